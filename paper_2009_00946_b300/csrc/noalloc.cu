// Layer reconstruction phi = W^{-1} c without any device allocation.
//
// Some callers cannot call cudaMalloc: a real-time control loop whose memory
// is reserved once at start-up and must not change while the loop runs (an
// allocation can block and synchronise the device), a plug-in that runs
// inside another framework which owns all device memory, or a process whose
// memory budget is already spent.  For them this file provides one entry
// point that computes the inverse db3 DWT of a stack of layers from
// caller-owned device buffers.  The column pass of each level needs an
// intermediate array; it lives in the file-scope array below, which every GPU
// that loads the library reserves once and keeps until the process exits.
//
// The first call on a device resolves the array's device address
// (cudaGetSymbolAddress) and caches it; make that first call before any
// stream capture.  All calls share the one array, so calls whose work
// overlaps on the GPU (different streams, or different host threads) race.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <mutex>

#include "debug.cuh"
#include "fewha.h"
#include "setup.h"

namespace fewha {
FEWHA_DBG_READER(dbg_read_noalloc)
}  // namespace fewha

using fewha::kDbgNoalloc;

namespace {

// 2^20 floats = 4 MiB of scratch: a stack of layers with at most this many
// coefficients in total (e.g. 35 layers of 128 x 128, or 16 of 256 x 256).
constexpr long kScratchFloats = 1L << 20;
constexpr int kMaxDevices = 64;

static __device__ __align__(256) float g_noalloc_scratch[kScratchFloats];

// Device address of the scratch array, resolved once per device.
float* g_scratch_ptr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mutex;

struct LayerStack {
    int L, Jmax, nmax;
    long total;   // coefficients of the stack (the source and destination length)
    int n[FEWHA_MAX_LAYERS];
    int J[FEWHA_MAX_LAYERS];
    int off[FEWHA_MAX_LAYERS];
    float h[6], g[6];
};

// inverse column pass of level j: x[i] = sum over taps t with (i - t) mod m
// even of h_t a_k + g_t d_k, k = ((i - t) mod m) / 2
__global__ void k_noalloc_inv_cols(LayerStack S, int j, const float* __restrict__ src, float* __restrict__ dst) {
    const int l = blockIdx.y;
    if (j > S.J[l]) return;
    const int n = S.n[l], m = n >> (j - 1), half = m >> 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    const int i = idx / m, x = idx - i * m;
    const float* s = src + S.off[l] + x;
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        const int r = ((i - t) % m + m) % m;
        if (r & 1) continue;
        const int k = r >> 1;
        if (!FEWHA_IN(S.off[l] + (long)(half + k) * n + x, S.total, 1, kDbgNoalloc)) continue;
        acc += S.h[t] * s[(long)k * n] + S.g[t] * s[(long)(half + k) * n];
    }
    if (FEWHA_IN(S.off[l] + (long)i * n + x, S.total, 1, kDbgNoalloc)) dst[S.off[l] + (long)i * n + x] = acc;
}

// inverse row pass of level j
__global__ void k_noalloc_inv_rows(LayerStack S, int j, const float* __restrict__ src, float* __restrict__ dst) {
    const int l = blockIdx.y;
    if (j > S.J[l]) return;
    const int n = S.n[l], m = n >> (j - 1), half = m >> 1;
    const int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= m * m) return;
    const int y = idx / m, i = idx - y * m;
    const float* s = src + S.off[l] + (long)y * n;
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < 6; ++t) {
        const int r = ((i - t) % m + m) % m;
        if (r & 1) continue;
        const int k = r >> 1;
        if (!FEWHA_IN(S.off[l] + (long)y * n + half + k, S.total, 1, kDbgNoalloc)) continue;
        acc += S.h[t] * s[k] + S.g[t] * s[half + k];
    }
    if (FEWHA_IN(S.off[l] + (long)y * n + i, S.total, 1, kDbgNoalloc)) dst[S.off[l] + (long)y * n + i] = acc;
}

int fail(char* errbuf, int errlen, int code, const char* msg) {
    if (errbuf && errlen > 0) snprintf(errbuf, errlen, "%s", msg);
    return code;
}

}  // namespace

extern "C" int fewha_layers_noalloc(const float* coeffs, float* layers, int n_layers, const int* n_side,
                                    const int* levels, void* stream, char* errbuf, int errlen) {
    if (errbuf && errlen > 0) errbuf[0] = '\0';
    if (!coeffs || !layers || !n_side || !levels)
        return fail(errbuf, errlen, FEWHA_ERR_ARG, "null pointer argument");
    if (coeffs == layers) return fail(errbuf, errlen, FEWHA_ERR_ARG, "coeffs and layers must not alias");
    if (n_layers < 1 || n_layers > FEWHA_MAX_LAYERS)
        return fail(errbuf, errlen, FEWHA_ERR_ARG, "n_layers must be in 1..64");
    LayerStack S;
    std::memset(&S, 0, sizeof S);
    S.L = n_layers;
    long total = 0;
    for (int l = 0; l < n_layers; ++l) {
        const int n = n_side[l], J = levels[l];
        if (n < 8 || n > 1024 || (n & (n - 1)))
            return fail(errbuf, errlen, FEWHA_ERR_ARG, "n_side must be a power of two in 8..1024");
        if (J < 1 || (n >> J) < 2) return fail(errbuf, errlen, FEWHA_ERR_ARG, "levels must satisfy 1 <= J, n >> J >= 2");
        S.n[l] = n;
        S.J[l] = J;
        S.off[l] = (int)total;
        S.Jmax = J > S.Jmax ? J : S.Jmax;
        S.nmax = n > S.nmax ? n : S.nmax;
        total += (long)n * n;
    }
    S.total = total;
    if (total > kScratchFloats) {
        char msg[160];
        snprintf(msg, sizeof msg, "%ld coefficients exceed the fixed scratch of %ld floats (4 MiB)", total,
                 kScratchFloats);
        return fail(errbuf, errlen, FEWHA_ERR_ARG, msg);
    }
    {
        // the copy and the level passes assume disjoint buffers
        const uintptr_t c0 = (uintptr_t)coeffs, c1 = c0 + (uintptr_t)total * sizeof(float);
        const uintptr_t y0 = (uintptr_t)layers, y1 = y0 + (uintptr_t)total * sizeof(float);
        if (c0 < y1 && y0 < c1) return fail(errbuf, errlen, FEWHA_ERR_ARG, "coeffs and layers must not overlap");
    }
    double h[6], g[6];
    fewha::db3_taps(h, g);
    for (int i = 0; i < 6; ++i) {
        S.h[i] = (float)h[i];
        S.g[i] = (float)g[i];
    }

    // once per device: the scratch array's device address (host code only
    // holds a stand-in for the symbol, never usable as a device pointer)
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) {
        cudaGetLastError();
        return fail(errbuf, errlen, FEWHA_ERR_CUDA, "no current CUDA device");
    }
    float* scratch = nullptr;
    {
        std::lock_guard<std::mutex> lock(g_scratch_mutex);
        if (!g_scratch_ptr[dev]) {
            void* p = nullptr;
            cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
            if (e != cudaSuccess || !p) {
                cudaGetLastError();
                return fail(errbuf, errlen, FEWHA_ERR_CUDA, "cudaGetSymbolAddress of the scratch array failed");
            }
            g_scratch_ptr[dev] = (float*)p;
        }
        scratch = g_scratch_ptr[dev];
    }

    // every scratch element a pass reads was written earlier in this call by
    // the previous pass, so nothing has to be cleared first
    cudaStream_t st = (cudaStream_t)stream;
    cudaError_t e = cudaMemcpyAsync(layers, coeffs, (size_t)total * sizeof(float), cudaMemcpyDeviceToDevice, st);
    for (int j = S.Jmax; j >= 1 && e == cudaSuccess; --j) {
        const int m = S.nmax >> (j - 1);
        const dim3 grid((m * m + 255) / 256, S.L);
        k_noalloc_inv_cols<<<grid, 256, 0, st>>>(S, j, layers, scratch);
        k_noalloc_inv_rows<<<grid, 256, 0, st>>>(S, j, scratch, layers);
        e = cudaGetLastError();
    }
    if (e != cudaSuccess) return fail(errbuf, errlen, FEWHA_ERR_CUDA, cudaGetErrorString(e));
    return FEWHA_OK;
}
