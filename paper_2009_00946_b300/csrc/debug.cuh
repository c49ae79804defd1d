// Bounds checks of the debug build (compiled in with -DFEWHA_DEBUG; the
// release library compiles every check to `true` and is unchanged).
//
// compute-sanitizer is not available where this library is tested, so the
// debug build checks, at every gather and scatter of the hot path, that the
// computed index lies inside the buffer it addresses: the global state and
// field vectors (against the instance's sizes) and the CTA's own or a cluster
// peer's shared memory (against the launch's dynamic shared-memory size).  A failed
// check records the site and index, counts the violation and SKIPS the
// access, so the kernel never touches memory outside its buffers; the host
// reads the record with fewha_debug_bounds.
//
// Each translation unit that includes this header has its own record (the
// library is built without relocatable device code); FEWHA_DBG_READER
// defines the host function that reads and clears it.
#pragma once
#include <cuda_runtime.h>

namespace fewha {

// check sites (the high 16 bits of the first-violation word)
enum DbgSite {
    kDbgNone = 0,
    kDbgWinSrc = 1,      // fused sensor tile: bilinear read of the layer cells (phi)
    kDbgWinDst = 2,      //   reserved (staged windows, no longer used)
    kDbgWinP = 3,        //   reserved (staged windows, no longer used)
    kDbgSlopes = 4,      // fused sensor tile: slope / mask index
    kDbgGtOut = 5,       // fused sensor tile: Gamma^T output node
    kDbgStgSrc = 6,      // fused layer phase: sensor field staged from psi
    kDbgStgDst = 7,      //   ... into shared memory
    kDbgPtRead = 8,      // fused layer phase: P^T gather read
    kDbgCascOwn = 9,     // level-stacked DWT: store into a row owner's shared memory
    kDbgCascCol = 10,    // level-stacked DWT: store into a column owner's shared memory
    kDbgCoef = 11,       // fused layer phase: owned coefficient index
    kDbgTT = 12,         // fused layer phase: tip-tilt correction node
    kDbgPhiOut = 13,     // fused layer phase: layer output
    kDbgStripe = 14,     // row-stripe DWT: peer row read
    kDbgTables = 15,     // fused: gather / interpolation table staging
    kDbgPlainP = 16,     // plain path: P gather from the layers
    kDbgPlainPT = 17,    // plain path: P^T gather from the sensor fields
    kDbgPlainGam = 18,   // plain path: Gamma / Gamma^T node or slope index
    kDbgFit = 19,        // fitting: sparse matrix column / vector index
    kDbgNoalloc = 20,    // fewha_layers_noalloc: coefficient index
    kDbgSites
};

#ifdef FEWHA_DEBUG
static __device__ unsigned long long g_dbg_first;   // site << 48 | (index & (2^48 - 1)) of the first violation
static __device__ unsigned long long g_dbg_count;

static __device__ __noinline__ void dbg_fail(int site, long long idx) {
    atomicCAS(&g_dbg_first, 0ull, ((unsigned long long)site << 48) | ((unsigned long long)idx & 0xffffffffffffull));
    atomicAdd(&g_dbg_count, 1ull);
}

// index i of an access of `width` elements inside [0, n)
static __device__ __forceinline__ bool dbg_in(long long i, long long n, int width, int site) {
    if (i >= 0 && i + width <= n) return true;
    dbg_fail(site, i);
    return false;
}

static __device__ __forceinline__ unsigned dbg_dyn_smem_bytes() {
    unsigned b;
    asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(b));
    return b;
}

// `bytes` bytes at the generic address p inside this CTA's dynamic shared
// memory (every checked shared-memory buffer lives there).  The offset is
// taken from the start of the dynamic region in the shared window: the
// window's own addresses do not start at 0 on this architecture.
static __device__ __forceinline__ bool dbg_in_smem(const void* p, int bytes, int site) {
    extern __shared__ __align__(16) unsigned char dbg_dyn_smem[];
    if (__isShared(p)) {
        const long long a =
            (long long)__cvta_generic_to_shared(p) - (long long)__cvta_generic_to_shared(dbg_dyn_smem);
        if (a >= 0 && a + bytes <= (long long)dbg_dyn_smem_bytes()) return true;
        dbg_fail(site, a);
    } else {
        dbg_fail(site, -1);
    }
    return false;
}

#define FEWHA_IN(i, n, width, site) ::fewha::dbg_in((long long)(i), (long long)(n), (width), (site))
#define FEWHA_IN_SMEM(p, bytes, site) ::fewha::dbg_in_smem((p), (bytes), (site))
#define FEWHA_DBG_READER(name)                                                              \
    int name(unsigned long long* first, unsigned long long* count) {                         \
        unsigned long long z = 0ull;                                                         \
        if (cudaMemcpyFromSymbol(first, g_dbg_first, sizeof(z)) != cudaSuccess) return -1;  \
        if (cudaMemcpyFromSymbol(count, g_dbg_count, sizeof(z)) != cudaSuccess) return -1;  \
        if (cudaMemcpyToSymbol(g_dbg_first, &z, sizeof(z)) != cudaSuccess) return -1;       \
        if (cudaMemcpyToSymbol(g_dbg_count, &z, sizeof(z)) != cudaSuccess) return -1;       \
        return 1;                                                                            \
    }
#else
#define FEWHA_IN(i, n, width, site) true
#define FEWHA_IN_SMEM(p, bytes, site) true
#define FEWHA_DBG_READER(name)                                           \
    int name(unsigned long long* first, unsigned long long* count) {      \
        *first = 0ull;                                                    \
        *count = 0ull;                                                    \
        return 0;                                                         \
    }
#endif

// host readers, one per translation unit with device code (1: debug build,
// 0: release build, -1: CUDA error)
int dbg_read_fused(unsigned long long* first, unsigned long long* count);
int dbg_read_solver(unsigned long long* first, unsigned long long* count);
int dbg_read_fitcg(unsigned long long* first, unsigned long long* count);
int dbg_read_noalloc(unsigned long long* first, unsigned long long* count);

}  // namespace fewha
