// Achievable L2 bandwidth of this GPU, measured with the library's own
// kernels: the denominator of the roofline of the fused frame kernel, whose
// working set (state vectors, sensor fields, tables: a few MB) stays resident
// in the 126 MB L2 for the whole frame, so the L2, not HBM, bounds its data
// movement.
//
// A buffer well below the L2 size is first written (it is then resident),
// then read -- or copied, its first half into its second -- `passes` times
// inside one launch, every access a 16-byte load or store that bypasses L1
// (ld.global.cg / st.global.cg), so each pass moves the whole buffer through
// the L2.  Each pass starts every thread at a different element (a rotation
// by pass), so no load can be reused from registers across passes.  Grids are
// a multiple of the SM count with four 512-thread CTAs per SM and eight
// independent 16-byte loads in flight per thread.
#include <cuda_runtime.h>

#include <algorithm>
#include <cstdio>
#include <vector>

#include "fewha.h"

namespace {

constexpr int kL2Threads = 512;
constexpr int kL2Unroll = 8;

__global__ void __launch_bounds__(kL2Threads) k_l2_fill(float4* buf, long n4) {
    for (long i = blockIdx.x * (long)blockDim.x + threadIdx.x; i < n4; i += (long)gridDim.x * blockDim.x)
        buf[i] = make_float4(1.f, 0.5f, 0.25f, 0.125f);
}

// Sum of every element, passes times over; the result is stored only when it
// is an impossible value (never), which keeps the loads alive.
__global__ void __launch_bounds__(kL2Threads) k_l2_read(const float4* __restrict__ buf, long n4, int passes,
                                                         float* sink) {
    const long nt = (long)gridDim.x * blockDim.x, t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    float acc = 0.f;
    for (int p = 0; p < passes; ++p) {
        const long rot = ((long)p * 7919L * 16L) % n4;
        for (long i0 = t; i0 < n4; i0 += nt * kL2Unroll) {
            float4 v[kL2Unroll];
#pragma unroll
            for (int u = 0; u < kL2Unroll; ++u) {
                long i = i0 + u * nt;
                if (i < n4) {
                    i += rot;
                    if (i >= n4) i -= n4;
                    v[u] = __ldcg(buf + i);
                } else {
                    v[u] = make_float4(0.f, 0.f, 0.f, 0.f);
                }
            }
#pragma unroll
            for (int u = 0; u < kL2Unroll; ++u) acc += (v[u].x + v[u].y) + (v[u].z + v[u].w);
        }
    }
    if (acc == -1.2345e-30f) sink[0] = acc;
}

// dst[i] = src[i] (halves of one buffer), passes times over.
__global__ void __launch_bounds__(kL2Threads) k_l2_copy(const float4* __restrict__ src, float4* __restrict__ dst,
                                                         long n4, int passes) {
    const long nt = (long)gridDim.x * blockDim.x, t = blockIdx.x * (long)blockDim.x + threadIdx.x;
    for (int p = 0; p < passes; ++p) {
        const long rot = ((long)p * 7919L * 16L) % n4;
        for (long i0 = t; i0 < n4; i0 += nt * kL2Unroll) {
            float4 v[kL2Unroll];
            long idx[kL2Unroll];
#pragma unroll
            for (int u = 0; u < kL2Unroll; ++u) {
                long i = i0 + u * nt;
                idx[u] = -1;
                if (i < n4) {
                    i += rot;
                    if (i >= n4) i -= n4;
                    idx[u] = i;
                    v[u] = __ldcg(src + i);
                }
            }
#pragma unroll
            for (int u = 0; u < kL2Unroll; ++u)
                if (idx[u] >= 0) __stcg(dst + idx[u], v[u]);
        }
    }
}

int fail(char* errbuf, int errlen, int code, const char* msg) {
    if (errbuf && errlen > 0) snprintf(errbuf, errlen, "%s", msg);
    return code;
}

}  // namespace

extern "C" int fewha_measure_l2(long bytes, int passes, int reps, double* read_gbs, double* copy_gbs, char* errbuf,
                                int errlen) {
    if (errbuf && errlen > 0) errbuf[0] = '\0';
    if (!read_gbs || !copy_gbs) return fail(errbuf, errlen, FEWHA_ERR_ARG, "null output pointer");
    if (bytes < (1L << 20) || bytes > (96L << 20) || (bytes % 256) != 0)
        return fail(errbuf, errlen, FEWHA_ERR_ARG, "bytes must be a multiple of 256 in 1 MiB .. 96 MiB");
    if (passes < 1 || passes > 10000 || reps < 1 || reps > 1000)
        return fail(errbuf, errlen, FEWHA_ERR_ARG, "passes in 1..10000, reps in 1..1000");
    int dev = 0, sms = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) !=
                                                  cudaSuccess) {
        cudaGetLastError();
        return fail(errbuf, errlen, FEWHA_ERR_CUDA, "no current CUDA device");
    }
    float4* buf = nullptr;
    float* sink = nullptr;
    cudaStream_t st = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaMalloc(&buf, (size_t)bytes);
    if (e == cudaSuccess) e = cudaMalloc(&sink, 256);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    const long n4 = bytes / 16, half4 = n4 / 2;
    const int grid = 4 * sms;
    std::vector<float> tr, tc;
    if (e == cudaSuccess) {
        k_l2_fill<<<grid, kL2Threads, 0, st>>>(buf, n4);
        k_l2_read<<<grid, kL2Threads, 0, st>>>(buf, n4, 2, sink);           // resident in L2 from here
        k_l2_copy<<<grid, kL2Threads, 0, st>>>(buf, buf + half4, half4, 2);
        e = cudaGetLastError();
    }
    for (int r = 0; r < reps && e == cudaSuccess; ++r) {
        float ms = 0.f;
        cudaEventRecord(e0, st);
        k_l2_read<<<grid, kL2Threads, 0, st>>>(buf, n4, passes, sink);
        cudaEventRecord(e1, st);
        e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        tr.push_back(ms);
        cudaEventRecord(e0, st);
        k_l2_copy<<<grid, kL2Threads, 0, st>>>(buf, buf + half4, half4, passes);
        cudaEventRecord(e1, st);
        if (e == cudaSuccess) e = cudaEventSynchronize(e1);
        if (e == cudaSuccess) e = cudaEventElapsedTime(&ms, e0, e1);
        tc.push_back(ms);
    }
    if (e == cudaSuccess) e = cudaGetLastError();
    if (e0) cudaEventDestroy(e0);
    if (e1) cudaEventDestroy(e1);
    if (st) cudaStreamDestroy(st);
    if (sink) cudaFree(sink);
    if (buf) cudaFree(buf);
    if (e != cudaSuccess) return fail(errbuf, errlen, FEWHA_ERR_CUDA, cudaGetErrorString(e));
    // the fastest repetition: bytes moved (read, or read + write) / time
    const double moved = (double)passes * (double)(n4 * 16);
    *read_gbs = moved / (*std::min_element(tr.begin(), tr.end()) * 1e-3) / 1e9;
    *copy_gbs = moved / (*std::min_element(tc.begin(), tc.end()) * 1e-3) / 1e9;
    return FEWHA_OK;
}
