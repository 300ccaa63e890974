// gs_noalloc.cu -- gs_bin_atoms_static: the atom cell list (stable counting
// sort) with its scratch in a fixed, file-scope device array, so that the
// call allocates no memory at all.
//
// Who needs it: callers that cannot let a library call cudaMalloc --
// programs that hand all device memory to their own allocator at start-up
// (a framework's caching pool, a fixed-budget service), or that cannot
// afford the implicit device-wide synchronisation a cudaMalloc/cudaFree may
// cause in the middle of their work.  They pass device buffers for the
// inputs and outputs; the temporaries live in g_bin_scratch below.
//
// Limits: at most GS_STATIC_MAX_ATOMS atoms and GS_STATIC_MAX_CELLS cells.
// The array (GS_STATIC_SCRATCH_BYTES, about 18 MB) is reserved on every GPU
// that loads the library, until the process exits.
//
// The atoms are ordered by cell with the same stable radix passes as the
// allocating entry point (gs_radix.cuh), so the time is bounded by the
// number of atoms however they crowd into cells.
//
// Sharing: every call uses the same array and it keeps the previous call's
// contents; the counters that must start at zero are cleared by each call.
// Calls whose work overlaps on the GPU (from two host threads, or on two
// streams without ordering) race on the array and give wrong results.
//
// Set-up: the first call on a device looks up the array's device address
// with cudaGetSymbolAddress (once per device, with that device current).
// Make that first call before any stream capture begins.
#include <mutex>

#include "gs_internal.cuh"
#include "gs_radix.cuh"

#define GS_STATIC_SCAN_THREADS 512
#define GS_STATIC_SCAN_TILE (GS_STATIC_SCAN_THREADS * 4)
// int32 words: counts [cells+1], cell of each atom [atoms], radix key and
// value buffers [atoms] each, digit histograms [256 * radix blocks] and the
// scan's tile sums (for the longer of counts and histograms)
#define GS_STATIC_RS_BLOCKS ((GS_STATIC_MAX_ATOMS + RS_TILE - 1) / RS_TILE)
#define GS_STATIC_TILES ((GS_STATIC_MAX_CELLS + 1 + GS_STATIC_SCAN_TILE - 1) / GS_STATIC_SCAN_TILE)
#define GS_STATIC_SCRATCH_WORDS \
    ((GS_STATIC_MAX_CELLS + 1) + 3 * GS_STATIC_MAX_ATOMS + 256 * GS_STATIC_RS_BLOCKS + GS_STATIC_TILES + 64)
#define GS_STATIC_SCRATCH_BYTES (4ull * GS_STATIC_SCRATCH_WORDS)

static __device__ __align__(256) int32_t g_bin_scratch[GS_STATIC_SCRATCH_WORDS];

static std::mutex g_static_mu;
static int32_t *g_static_ptr[64];

// once per device, with that device current: the array's device address
static int static_scratch(int32_t **out)
{
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return gs_fail_cuda(e, "cudaGetDevice", __FILE__, __LINE__);
    if (dev < 0 || dev >= 64) return gs_fail(GS_ERR_ARG, "device index out of range");
    std::lock_guard<std::mutex> lk(g_static_mu);
    if (!g_static_ptr[dev]) {
        void *p = nullptr;
        e = cudaGetSymbolAddress(&p, g_bin_scratch);
        if (e != cudaSuccess) return gs_fail_cuda(e, "cudaGetSymbolAddress(g_bin_scratch)", __FILE__, __LINE__);
        g_static_ptr[dev] = (int32_t *)p;
    }
    *out = g_static_ptr[dev];
    return GS_OK;
}

__global__ void k_static_zero(int32_t *a, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        a[i] = 0;
}

__global__ void k_static_count(const double *__restrict__ xyz, int64_t n, double ox, double oy, double oz, double inv,
                               int cx, int cy, int cz, int32_t *__restrict__ cell_of_atom, int32_t *__restrict__ counts)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int c3[3];
    const double o[3] = {ox, oy, oz};
    const int dim[3] = {cx, cy, cz};
    for (int a = 0; a < 3; a++) {
        double f = floor(__dmul_rn(__dsub_rn(xyz[3 * i + a], o[a]), inv));
        c3[a] = f < 0.0 ? 0 : (f >= (double)dim[a] ? dim[a] - 1 : (int)f);
    }
    int k = c3[0] + cx * (c3[1] + cy * c3[2]);
    cell_of_atom[i] = k;
    atomicAdd(&counts[k], 1);
}

// exclusive scan of int32 counts in place, tile totals in sums
__device__ __forceinline__ int32_t static_block_scan(int32_t v, int32_t *total)
{
    __shared__ int32_t wt[GS_STATIC_SCAN_THREADS / 32];
    int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    int32_t inc = v;
    for (int o = 1; o < 32; o <<= 1) {
        int32_t t = __shfl_up_sync(0xffffffffu, inc, o);
        if (lane >= o) inc += t;
    }
    if (lane == 31) wt[w] = inc;
    __syncthreads();
    if (w == 0) {
        int32_t t = lane < GS_STATIC_SCAN_THREADS / 32 ? wt[lane] : 0;
        for (int o = 1; o < 32; o <<= 1) {
            int32_t u = __shfl_up_sync(0xffffffffu, t, o);
            if (lane >= o) t += u;
        }
        if (lane < GS_STATIC_SCAN_THREADS / 32) wt[lane] = t;
    }
    __syncthreads();
    int32_t before = w ? wt[w - 1] : 0;
    *total = wt[GS_STATIC_SCAN_THREADS / 32 - 1];
    __syncthreads();
    return before + inc - v;
}

__global__ void k_static_tile_sums(const int32_t *__restrict__ v, int64_t n, int32_t *__restrict__ sums)
{
    int64_t base = (int64_t)blockIdx.x * GS_STATIC_SCAN_TILE + (int64_t)threadIdx.x * 4;
    int32_t s = 0;
    for (int i = 0; i < 4; i++)
        if (base + i < n) s += v[base + i];
    int32_t tot;
    static_block_scan(s, &tot);
    if (threadIdx.x == 0) sums[blockIdx.x] = tot;
}

// one block: exclusive scan of the tile sums (at most GS_STATIC_TILES values)
__global__ void k_static_scan_sums(int32_t *sums, int64_t ntiles)
{
    int32_t carry = 0;
    for (int64_t b = 0; b < ntiles; b += GS_STATIC_SCAN_THREADS) {
        int64_t i = b + threadIdx.x;
        int32_t v = i < ntiles ? sums[i] : 0;
        int32_t tot;
        int32_t ex = static_block_scan(v, &tot);
        if (i < ntiles) sums[i] = carry + ex;
        carry += tot;
    }
}

__global__ void k_static_tile_apply(int32_t *__restrict__ v, int64_t n, const int32_t *__restrict__ offs)
{
    int64_t base = (int64_t)blockIdx.x * GS_STATIC_SCAN_TILE + (int64_t)threadIdx.x * 4;
    int32_t loc[4], s = 0;
    for (int i = 0; i < 4; i++) {
        loc[i] = base + i < n ? v[base + i] : 0;
        s += loc[i];
    }
    int32_t tot;
    int32_t pre = static_block_scan(s, &tot) + offs[blockIdx.x];
    for (int i = 0; i < 4; i++) {
        if (base + i < n) v[base + i] = pre;
        pre += loc[i];
    }
}

__global__ void k_static_starts(const int32_t *__restrict__ start, int64_t ncell, int32_t *__restrict__ cell_start)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= ncell) cell_start[k] = start[k];
}

// exclusive scan of m int32 values in place (tile sums in sums)
static void static_scan(int32_t *v, int64_t m, int32_t *sums, cudaStream_t st)
{
    int64_t tiles = (m + GS_STATIC_SCAN_TILE - 1) / GS_STATIC_SCAN_TILE;
    k_static_tile_sums<<<(unsigned)tiles, GS_STATIC_SCAN_THREADS, 0, st>>>(v, m, sums);
    k_static_scan_sums<<<1, GS_STATIC_SCAN_THREADS, 0, st>>>(sums, tiles);
    k_static_tile_apply<<<(unsigned)tiles, GS_STATIC_SCAN_THREADS, 0, st>>>(v, m, sums);
}

// device (or managed) memory of the current device
static bool is_device_ptr(const void *p, int dev)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return (a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged) && a.device == dev;
}

extern "C" int gs_bin_atoms_static(const double *atoms, int64_t n_atoms, double cell_size, const double *origin,
                                   const int64_t *dims, int32_t *cell_start, int32_t *atom_perm, void *stream)
{
    if (!atoms || !origin || !dims || !cell_start || !atom_perm || !(cell_size > 0))
        return gs_fail(GS_ERR_ARG, "gs_bin_atoms_static: NULL pointer or non-positive cell size");
    if (n_atoms <= 0 || n_atoms > GS_STATIC_MAX_ATOMS)
        return gs_fail(GS_ERR_ARG, "gs_bin_atoms_static: n_atoms must be in [1, %d]", GS_STATIC_MAX_ATOMS);
    int64_t ncell = 1;
    int cd[3];
    for (int a = 0; a < 3; a++) {
        if (dims[a] <= 0 || dims[a] > GS_STATIC_MAX_CELLS)
            return gs_fail(GS_ERR_ARG, "gs_bin_atoms_static: each of dims must be in [1, %d]", GS_STATIC_MAX_CELLS);
        cd[a] = (int)dims[a];
        ncell *= dims[a];
        if (ncell > GS_STATIC_MAX_CELLS)
            return gs_fail(GS_ERR_ARG, "gs_bin_atoms_static: at most %d cells", GS_STATIC_MAX_CELLS);
    }
    int dev = 0;
    cudaError_t de = cudaGetDevice(&dev);
    if (de != cudaSuccess) return gs_fail_cuda(de, "cudaGetDevice", __FILE__, __LINE__);
    if (!is_device_ptr(atoms, dev) || !is_device_ptr(cell_start, dev) || !is_device_ptr(atom_perm, dev))
        return gs_fail(GS_ERR_ARG, "gs_bin_atoms_static: atoms, cell_start and atom_perm must be device memory of "
                                   "the current device");
    int32_t *scr = nullptr;
    int rc = static_scratch(&scr);
    if (rc) return rc;
    const int64_t nblk = (n_atoms + RS_TILE - 1) / RS_TILE;
    int32_t *counts = scr;                       // [ncell + 1]
    int32_t *coa = counts + (ncell + 1);         // [n_atoms]
    int32_t *kb = coa + n_atoms;                 // [n_atoms]
    int32_t *vb = kb + n_atoms;                  // [n_atoms]
    int32_t *hist = vb + n_atoms;                // [256 * nblk]
    int32_t *sums = hist + 256 * nblk;           // [tiles]
    cudaStream_t st = (cudaStream_t)stream;
    const unsigned nb = (unsigned)((n_atoms + 255) / 256);
    int64_t nz = ncell + 1;
    k_static_zero<<<(unsigned)((nz + 255) / 256 < 4096 ? (nz + 255) / 256 : 4096), 256, 0, st>>>(counts, nz);
    k_static_count<<<nb, 256, 0, st>>>(atoms, n_atoms, origin[0], origin[1], origin[2], 1.0 / cell_size, cd[0], cd[1],
                                       cd[2], coa, counts);
    static_scan(counts, ncell + 1, sums, st);
    k_static_starts<<<(unsigned)((ncell + 1 + 255) / 256), 256, 0, st>>>(counts, ncell, cell_start);
    // stable radix passes on the cell index; the last writes atom_perm
    const int passes = rs_passes(ncell);
    if (passes == 0) k_rs_iota<<<nb, 256, 0, st>>>(atom_perm, n_atoms);
    int32_t *kbuf[2] = {kb, coa};
    int32_t *vbuf[2];
    vbuf[(passes - 1) & 1] = atom_perm;
    vbuf[passes & 1] = vb;
    for (int p = 0; p < passes; p++) {
        const int32_t *kin = p == 0 ? coa : kbuf[(p - 1) & 1];
        int32_t *kout = p == passes - 1 ? nullptr : kbuf[p & 1];
        const int32_t *vin = p == 0 ? nullptr : vbuf[(p - 1) & 1];
        k_rs_hist<int32_t><<<(unsigned)nblk, RS_THREADS, 0, st>>>(kin, n_atoms, 8 * p, hist, nblk);
        static_scan(hist, 256 * nblk, sums, st);
        k_rs_scatter<int32_t><<<(unsigned)nblk, RS_THREADS, 0, st>>>(kin, vin, n_atoms, 8 * p, hist, nblk, kout,
                                                                    vbuf[p & 1]);
    }
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return gs_fail_cuda(e, "gs_bin_atoms_static launch", __FILE__, __LINE__);
    e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return gs_fail_cuda(e, "gs_bin_atoms_static", __FILE__, __LINE__);
    return GS_OK;
}
