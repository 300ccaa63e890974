// gs_scan.cu -- exclusive prefix sums for stream compaction (level lists,
// vertex and point ownership), error helpers and workspace allocation.
#include <cstdarg>
#include <cstdio>
#include <cstring>

#include "gs_host.cuh"

static thread_local char g_last_error[512] = "";

int gs_fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_last_error, sizeof(g_last_error), fmt, ap);
    va_end(ap);
    return code;
}

int gs_fail_cuda(cudaError_t e, const char *what, const char *file, int line)
{
    const char *f = strrchr(file, '/');
    if (e == cudaErrorTimeout) {
        gs_fail(GS_ERR_TIMEOUT, "%s: host wait passed its deadline (%s:%d)", what, f ? f + 1 : file, line);
        return GS_ERR_TIMEOUT;
    }
    gs_fail(e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA, "%s failed: %s (%s:%d)", what,
            cudaGetErrorString(e), f ? f + 1 : file, line);
    return e == cudaErrorMemoryAllocation ? GS_ERR_OOM : GS_ERR_CUDA;
}

extern "C" const char *gs_last_error(void) { return g_last_error; }

// per host thread: a call runs on one thread, so the difference over the
// call counts exactly its own launches even when calls run concurrently
static thread_local long long g_launches = 0;
void gs_count_launch(void) { g_launches++; }
long long gs_launch_count(void) { return g_launches; }

int gs_alloc(void **p, size_t bytes, cudaStream_t st)
{
    *p = nullptr;
    if (gs_fault_alloc()) return gs_fail(GS_ERR_OOM, "device allocation failed (injected by GS_FAULT)");
    if (bytes == 0) bytes = 16;
    cudaError_t e = cudaMallocAsync(p, bytes, st);
    if (e != cudaSuccess) {
        *p = nullptr;
        return gs_fail_cuda(e, "cudaMallocAsync", __FILE__, __LINE__);
    }
    return GS_OK;
}

void gs_free(void *p, cudaStream_t st)
{
    if (p) cudaFreeAsync(p, st);
}

// ---------------------------------------------------------------- scan
// Three phases: per-block totals, scan of the totals (recursively), and a
// per-block scan that adds the block's offset.  Each block covers
// SCAN_THREADS * SCAN_ITEMS consecutive values.
#define SCAN_THREADS 512
#define SCAN_ITEMS 8
#define SCAN_TILE (SCAN_THREADS * SCAN_ITEMS)

__device__ __forceinline__ int64_t warp_incl_scan(int64_t v)
{
    for (int o = 1; o < 32; o <<= 1) {
        int64_t t = __shfl_up_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) >= o) v += t;
    }
    return v;
}

// exclusive block scan of one value per thread; returns the block total in *total
__device__ __forceinline__ int64_t block_excl_scan(int64_t v, int64_t *total)
{
    __shared__ int64_t warp_tot[SCAN_THREADS / 32];
    int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int64_t inc = warp_incl_scan(v);
    if (lane == 31) warp_tot[wid] = inc;
    __syncthreads();
    if (wid == 0) {
        int64_t t = lane < SCAN_THREADS / 32 ? warp_tot[lane] : 0;
        t = warp_incl_scan(t);
        if (lane < SCAN_THREADS / 32) warp_tot[lane] = t;
    }
    __syncthreads();
    int64_t before = wid > 0 ? warp_tot[wid - 1] : 0;
    *total = warp_tot[SCAN_THREADS / 32 - 1];
    __syncthreads();
    return before + inc - v;
}

__global__ void k_scan_tile_sums(const int64_t *__restrict__ v, int64_t n, int64_t *__restrict__ sums)
{
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++)
        if (base + i < n) s += v[base + i];
    int64_t tot;
    block_excl_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

__global__ void k_scan_tile_apply(int64_t *__restrict__ v, int64_t n, const int64_t *__restrict__ offs)
{
    int64_t base = (int64_t)blockIdx.x * SCAN_TILE + (int64_t)threadIdx.x * SCAN_ITEMS;
    int64_t loc[SCAN_ITEMS];
    int64_t s = 0;
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        loc[i] = base + i < n ? v[base + i] : 0;
        s += loc[i];
    }
    int64_t tot;
    int64_t pre = block_excl_scan(s, &tot) + (offs ? offs[blockIdx.x] : 0);
#pragma unroll
    for (int i = 0; i < SCAN_ITEMS; i++) {
        if (base + i < n) v[base + i] = pre;
        pre += loc[i];
    }
}

__global__ void k_scan_total(const int64_t *v, const int64_t *orig_last, int64_t n, int64_t *total)
{
    // total = exclusive[n-1] + original value at n-1
    *total = n > 0 ? v[n - 1] + *orig_last : 0;
}

int gs_scan_i64(int64_t *d_vals, int64_t n, int64_t *d_total, cudaStream_t st)
{
    if (n <= 0) {
        if (d_total) GS_CHECK(cudaMemsetAsync(d_total, 0, sizeof(int64_t), st));
        return GS_OK;
    }
    int64_t *last = nullptr;
    int rc = gs_alloc((void **)&last, sizeof(int64_t), st);
    if (rc) return rc;
    GS_CHECK(cudaMemcpyAsync(last, d_vals + (n - 1), sizeof(int64_t), cudaMemcpyDeviceToDevice, st));
    int64_t tiles = (n + SCAN_TILE - 1) / SCAN_TILE;
    if (tiles == 1) {
        GS_LAUNCH(k_scan_tile_apply, 1, SCAN_THREADS, 0, st)(d_vals, n, nullptr);
    } else {
        int64_t *sums = nullptr;
        rc = gs_alloc((void **)&sums, sizeof(int64_t) * (size_t)tiles, st);
        if (rc) { gs_free(last, st); return rc; }
        GS_LAUNCH(k_scan_tile_sums, (unsigned)tiles, SCAN_THREADS, 0, st)(d_vals, n, sums);
        rc = gs_scan_i64(sums, tiles, nullptr, st);
        if (rc) { gs_free(sums, st); gs_free(last, st); return rc; }
        GS_LAUNCH(k_scan_tile_apply, (unsigned)tiles, SCAN_THREADS, 0, st)(d_vals, n, sums);
        gs_free(sums, st);
    }
    if (d_total) GS_LAUNCH(k_scan_total, 1, 1, 0, st)(d_vals, last, n, d_total);
    gs_free(last, st);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// ---------------------------------------------------------------- host copies
// Copies between device memory and page-locked host memory run as a kernel
// on the host buffer's device mapping (16-byte loads and stores, grid a
// multiple of the SM count), so a large mesh leaves the device at the rate of
// the host link without a staging step; other host memory (pageable,
// unregistered) and unaligned buffers take cudaMemcpyAsync.
__global__ void __launch_bounds__(256) k_copy16(int4 *__restrict__ dst, const int4 *__restrict__ src, int64_t n16)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n16; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// the host buffer's device address when it is page-locked and mapped, else null
static void *mapped_host(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return nullptr;
    }
    return a.type == cudaMemoryTypeHost ? a.devicePointer : nullptr;
}

int gs_host_kind(const void *p)
{
    cudaPointerAttributes a;
    if (!p) return -1;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
        cudaGetLastError();
        return 2;
    }
    if (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) return 0;
    if (a.type == cudaMemoryTypeHost) return a.devicePointer ? 1 : 2;
    return 2;
}

static int copy_mapped(void *dst_dev, const void *src_dev, size_t bytes, cudaStream_t st)
{
    const int64_t n16 = (int64_t)(bytes / 16);
    if (n16 > 0) {
        int64_t blocks = (n16 + 255) / 256;
        if (blocks > 152 * 8) blocks = 152 * 8;
        GS_LAUNCH(k_copy16, (unsigned)blocks, 256, 0, st)((int4 *)dst_dev, (const int4 *)src_dev, n16);
    }
    const size_t tail = bytes - 16 * (size_t)n16;
    if (tail)
        GS_CHECK(cudaMemcpyAsync((char *)dst_dev + 16 * n16, (const char *)src_dev + 16 * n16, tail,
                                 cudaMemcpyDefault, st));
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

int gs_copy_to_host(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    if (!bytes) return GS_OK;
    void *dd = mapped_host(dst);
    if (dd && ((uintptr_t)dd % 16) == 0 && ((uintptr_t)src % 16) == 0) return copy_mapped(dd, src, bytes, st);
    GS_CHECK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    return GS_OK;
}

int gs_copy_from_host(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    if (!bytes) return GS_OK;
    void *sd = mapped_host(src);
    if (sd && ((uintptr_t)sd % 16) == 0 && ((uintptr_t)dst % 16) == 0) return copy_mapped(dst, sd, bytes, st);
    GS_CHECK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyDefault, st));
    return GS_OK;
}
