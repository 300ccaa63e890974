// gs_internal.cuh -- shared device helpers of the GB300 Gaussian-surface
// mesher (internal to the library; not part of the C ABI).
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>

#include "../../include/gsmesh.h"

// ---------------------------------------------------------------- keys
// bits 0..17 x, 18..35 y, 36..53 z, 54..58 type, 59..63 level
#define GK_BITS 18
#define GK_MASK 0x3FFFFull
#define GT_CUBE 30u
#define GT_VERT 31u

__host__ __device__ __forceinline__ uint64_t gk_make(uint64_t x, uint64_t y, uint64_t z, unsigned type,
                                                     unsigned level)
{
    return x | (y << 18) | (z << 36) | ((uint64_t)type << 54) | ((uint64_t)level << 59);
}
__host__ __device__ __forceinline__ int64_t gk_x(uint64_t k) { return (int64_t)(k & GK_MASK); }
__host__ __device__ __forceinline__ int64_t gk_y(uint64_t k) { return (int64_t)((k >> 18) & GK_MASK); }
__host__ __device__ __forceinline__ int64_t gk_z(uint64_t k) { return (int64_t)((k >> 36) & GK_MASK); }
__host__ __device__ __forceinline__ unsigned gk_level(uint64_t k) { return (unsigned)(k >> 59); }
__host__ __device__ __forceinline__ unsigned gk_type(uint64_t k) { return (unsigned)((k >> 54) & 31u); }

// ---------------------------------------------------------------- status word
// Kernels never trap: they set bits in a device status word and return.
#define GS_ST_CAPACITY 1u   // a fixed-size buffer or hash table overflowed
#define GS_ST_LOOP 2u       // a bounded loop hit its iteration limit
#define GS_ST_INPUT 4u      // non-finite or negative input
#define GS_ST_LOOKUP 8u     // a key that must exist was not found

// ---------------------------------------------------------------- decisions
#define DEC_DISCARD 0
#define DEC_ACCEPT 1
#define DEC_SPLIT 2
#define DEC_FORCED 3
#define DEC_INVALID 255

// ---------------------------------------------------------------- problem
struct GsProblem {
    int64_t n;           // atoms
    double D, c, KD;     // KD = -ln(cutoff_rel c) / D
    double precision;
    double min_edge;
    int max_depth;
    int order;           // GS_ORDER_*: decision order of steps 2 and 3 (FP64 form)
    int norm;            // GS_NORM_*: size of the higher-order coefficients (FP64 form)
    double origin[3];
    int64_t nroot[3];
    double pad;          // largest cutoff radius
    // cell list over the same origin
    double cell;         // cell edge
    double inv_cell;
    int cdim[3];
    // atoms in cell order (SoA)
    const double *ax, *ay, *az, *ar, *aR2, *aw;   // centre, radius, cutoff^2, exp(D r^2)
    const float *fx, *fy, *fz;                   // centres relative to their cell's lower corner (FP32)
    const float *hx, *lx, *hy, *ly, *hz, *lz;    // centre - origin as a two-float sum hi + lo
    const float *fw;                             // exp(D r^2) in FP32
    const float *fR2;                            // cutoff^2 in FP32 (prefilters only)
    const float *fr2;                            // r^2 in FP32
    const float *lr2;                            // r^2 - fr2 (r^2 = fr2 + lr2 to ~1e-14 relative)
    float cell_f, inv_cell_f, pad_f;             // FP32 copies for candidate enumeration
    int lat_exact_f32;                           // lattice coordinates (index * spacing) are exact in FP32
    const int32_t *cell_start;                   // [ncell + 1]
    // nullable: counts of decisions whose margin is below 1e-10 relative
    // ([0] bound test, [1] precision test, [2] rank rule, [3] vertex sign)
    unsigned long long *near;
};
#define GS_NEAR_REL 1e-10

// cube edge at level l (exact power-of-two scaling)
__host__ __device__ __forceinline__ double gs_h(const GsProblem &P, int l)
{
    return ldexp(P.min_edge, P.max_depth - l);
}
// world coordinate of lattice index i at level l on axis a: origin + i*h, no contraction
__device__ __forceinline__ double gs_lat(const GsProblem &P, int a, int64_t i, int l)
{
    return __dadd_rn(P.origin[a], __dmul_rn((double)i, gs_h(P, l)));
}

// squared distance from x to [lo,hi] along one axis, then summed x,y,z
__device__ __forceinline__ double gs_axis_gap(double lo, double hi, double x)
{
    double d = 0.0;
    if (__dsub_rn(lo, x) > 0.0) d = __dsub_rn(lo, x);
    else if (__dsub_rn(x, hi) > 0.0) d = __dsub_rn(x, hi);
    return d;
}
__device__ __forceinline__ double gs_box_d2(const double *lo, const double *hi, double x, double y, double z)
{
    double dx = gs_axis_gap(lo[0], hi[0], x), dy = gs_axis_gap(lo[1], hi[1], y), dz = gs_axis_gap(lo[2], hi[2], z);
    return __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
}

// Candidate cell rows around the box [lo, hi] (coordinates relative to the
// origin) grown by the largest cutoff radius, enumerated in FP32 -- GB300
// issues FP64 at 1/64 of the FP32 rate, so the per-row bookkeeping must not
// use it.  The 1e-3 A margins make the enumeration conservative: every atom
// within the cutoff of the box lies in a visited row; membership itself is
// decided by the caller.  body(begin, end, row, x0) gets each row's atom range.
template <typename F>
__device__ __forceinline__ void gs_for_rows(const GsProblem &P, const float *lo, const float *hi, F body)
{
    const float cs = P.cell_f, inv = P.inv_cell_f, pad = P.pad_f + 1e-3f;
    int c0[3], c1[3];
    for (int a = 0; a < 3; a++) {
        float f0 = floorf((lo[a] - pad) * inv), f1 = floorf((hi[a] + pad) * inv);
        f0 = fminf(fmaxf(f0, 0.f), (float)(P.cdim[a] - 1));
        f1 = fminf(fmaxf(f1, 0.f), (float)(P.cdim[a] - 1));
        c0[a] = (int)f0;
        c1[a] = (int)f1;
    }
    const float pad2 = pad * pad;
    for (int cz = c0[2]; cz <= c1[2]; cz++) {
        float zlo = cz * cs;
        float gz = fmaxf(0.f, fmaxf(zlo - hi[2], lo[2] - (zlo + cs)));
        if (gz * gz > pad2) continue;
        for (int cy = c0[1]; cy <= c1[1]; cy++) {
            float ylo = cy * cs;
            float gy = fmaxf(0.f, fmaxf(ylo - hi[1], lo[1] - (ylo + cs)));
            float rem2 = pad2 - gy * gy - gz * gz;
            if (rem2 < 0.f) continue;
            float rem = sqrtf(rem2) + 1e-3f;
            float f0 = fmaxf(floorf((lo[0] - rem) * inv), (float)c0[0]);
            float f1 = fminf(floorf((hi[0] + rem) * inv), (float)c1[0]);
            int x0 = (int)f0, x1 = (int)f1;
            if (x0 > x1) continue;
            int64_t row = (int64_t)P.cdim[0] * (cy + (int64_t)P.cdim[1] * cz);
            body(P.cell_start[row + x0], P.cell_start[row + x1 + 1], row, x0);
        }
    }
}

// Warp-cooperative form of gs_for_rows: the lanes compute the (y, z) rows in
// parallel (32 at a time), a warp scan concatenates their atom ranges, and
// chunk(i) is called by all lanes with one candidate atom index per lane
// (-1 past the end), 32 candidates per call.  Same rows and ranges as
// gs_for_rows; all lanes must call it with the same box.
template <typename F>
__device__ __forceinline__ void gs_warp_candidates(const GsProblem &P, const float *lo, const float *hi, int lane,
                                                   F chunk)
{
    const unsigned full = 0xffffffffu;
    const float cs = P.cell_f, inv = P.inv_cell_f, pad = P.pad_f + 1e-3f;
    int c0[3], c1[3];
    for (int a = 0; a < 3; a++) {
        float f0 = floorf((lo[a] - pad) * inv), f1 = floorf((hi[a] + pad) * inv);
        f0 = fminf(fmaxf(f0, 0.f), (float)(P.cdim[a] - 1));
        f1 = fminf(fmaxf(f1, 0.f), (float)(P.cdim[a] - 1));
        c0[a] = (int)f0;
        c1[a] = (int)f1;
    }
    const float pad2 = pad * pad;
    const int ny = c1[1] - c0[1] + 1, nz = c1[2] - c0[2] + 1, nrows = ny * nz;
    for (int r0 = 0; r0 < nrows; r0 += 32) {
        const int r = r0 + lane;
        int b = 0, len = 0;
        if (r < nrows) {
            const int cy = c0[1] + r % ny, cz = c0[2] + r / ny;
            float zlo = cz * cs;
            float gz = fmaxf(0.f, fmaxf(zlo - hi[2], lo[2] - (zlo + cs)));
            float ylo = cy * cs;
            float gy = fmaxf(0.f, fmaxf(ylo - hi[1], lo[1] - (ylo + cs)));
            float rem2 = pad2 - gy * gy - gz * gz;
            if (gz * gz <= pad2 && rem2 >= 0.f) {
                float rem = sqrtf(rem2) + 1e-3f;
                float f0 = fmaxf(floorf((lo[0] - rem) * inv), (float)c0[0]);
                float f1 = fminf(floorf((hi[0] + rem) * inv), (float)c1[0]);
                int x0 = (int)f0, x1 = (int)f1;
                if (x0 <= x1) {
                    int64_t row = (int64_t)P.cdim[0] * (cy + (int64_t)P.cdim[1] * cz);
                    b = P.cell_start[row + x0];
                    len = P.cell_start[row + x1 + 1] - b;
                }
            }
        }
        int incl = len;
#pragma unroll
        for (int o = 1; o < 32; o <<= 1) {
            int v = __shfl_up_sync(full, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(full, incl, 31), excl = incl - len;
        for (int g0 = 0; g0 < total; g0 += 32) {
            const int g = g0 + lane;
            // the last row whose range starts at or before g
            int src = 0;
#pragma unroll
            for (int step = 16; step > 0; step >>= 1) {
                int e = __shfl_sync(full, excl, src + step);
                if (e <= g) src += step;
            }
            const int bs = __shfl_sync(full, b, src), es = __shfl_sync(full, excl, src);
            chunk(g < total ? bs + (g - es) : -1);
        }
    }
}

// ---------------------------------------------------------------- exp (FP64)
// 2^x by the hardware approximation (ex2.approx, relative error <= 2^-22,
// results below 2^-126 flushed to zero).  The FP32 factors and terms it
// serves stay far above that range: their arguments are bounded by the
// cutoff, and a weight exp(D r^2) large enough to reach it overflows FP32
// first.
__device__ __forceinline__ float gs_ex2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}

// exp(x) for |x| <= 700 by Tang's table-driven method (ACM TOMS 15, 1989):
// x = (32 m + j) ln2/32 + r with |r| <= ln2/64 (Cody-Waite reduction, ln2/32
// split so that k * GS_L1 is exact for |k| < 2^15), exp(r) - 1 by its degree-6
// Taylor polynomial (truncation below 4e-18), then 2^(j/32) from a table and
// 2^m into the exponent field.  Error within 2 ulp; no special cases.
static __device__ const double gs_exp_tab[32] = {
    0x1.0000000000000p+0, 0x1.059b0d3158574p+0, 0x1.0b5586cf9890fp+0, 0x1.11301d0125b51p+0,
    0x1.172b83c7d517bp+0, 0x1.1d4873168b9aap+0, 0x1.2387a6e756238p+0, 0x1.29e9df51fdee1p+0,
    0x1.306fe0a31b715p+0, 0x1.371a7373aa9cbp+0, 0x1.3dea64c123422p+0, 0x1.44e086061892dp+0,
    0x1.4bfdad5362a27p+0, 0x1.5342b569d4f82p+0, 0x1.5ab07dd485429p+0, 0x1.6247eb03a5585p+0,
    0x1.6a09e667f3bcdp+0, 0x1.71f75e8ec5f74p+0, 0x1.7a11473eb0187p+0, 0x1.82589994cce13p+0,
    0x1.8ace5422aa0dbp+0, 0x1.93737b0cdc5e5p+0, 0x1.9c49182a3f090p+0, 0x1.a5503b23e255dp+0,
    0x1.ae89f995ad3adp+0, 0x1.b7f76f2fb5e47p+0, 0x1.c199bdd85529cp+0, 0x1.cb720dcef9069p+0,
    0x1.d5818dcfba487p+0, 0x1.dfc97337b9b5fp+0, 0x1.ea4afa2a490dap+0, 0x1.f50765b6e4540p+0};

__device__ __forceinline__ double gs_exp(double x)
{
    const double inv = 0x1.71547652b82fep+5;      // 32 / ln 2
    const double L1 = 0x1.62e42fefa0000p-6;       // ln 2 / 32, leading 37 bits
    const double L2 = 0x1.cf79abc9e3b3ap-45;      // ln 2 / 32 - L1
    const double shifter = 0x1.8p+52;             // rounds to an integer in the low word
    double t = fma(x, inv, shifter);
    const int k = __double2loint(t);
    const double kd = t - shifter;
    double r = fma(-kd, L1, x);
    r = fma(-kd, L2, r);
    double p = fma(r, 1.0 / 720.0, 1.0 / 120.0);
    p = fma(r, p, 1.0 / 24.0);
    p = fma(r, p, 1.0 / 6.0);
    p = fma(r, p, 0.5);
    p = fma(r * r, p, r);                         // exp(r) - 1
    const double s = __ldg(&gs_exp_tab[k & 31]);
    const double y = fma(s, p, s);
    return __hiloint2double(__double2hiint(y) + ((k >> 5) << 20), __double2loint(y));
}

// ---------------------------------------------------------------- hashing
#define GS_EMPTY 0xFFFFFFFFFFFFFFFFull
__host__ __device__ __forceinline__ uint64_t gs_mix(uint64_t k)
{
    k ^= k >> 33;
    k *= 0xff51afd7ed558ccdull;
    k ^= k >> 33;
    k *= 0xc4ceb9fe1a85ec53ull;
    k ^= k >> 33;
    return k;
}

struct GsHash {
    uint64_t *keys;   // capacity, GS_EMPTY when free
    uint64_t *vals;   // capacity
    uint64_t mask;    // capacity - 1 (power of two)
};

// insert key; returns slot (or -1 when full); the slot's value is left alone
__device__ __forceinline__ int64_t gs_hash_insert(const GsHash &H, uint64_t key, unsigned *status)
{
    uint64_t s = gs_mix(key) & H.mask;
    for (uint64_t probe = 0; probe <= H.mask; probe++) {
        unsigned long long prev = atomicCAS((unsigned long long *)&H.keys[s], (unsigned long long)GS_EMPTY,
                                            (unsigned long long)key);
        if (prev == GS_EMPTY || prev == key) return (int64_t)s;
        s = (s + 1) & H.mask;
    }
    atomicOr(status, GS_ST_CAPACITY);
    return -1;
}
__device__ __forceinline__ int64_t gs_hash_find(const GsHash &H, uint64_t key)
{
    uint64_t s = gs_mix(key) & H.mask;
    for (uint64_t probe = 0; probe <= H.mask; probe++) {
        uint64_t k = H.keys[s];
        if (k == key) return (int64_t)s;
        if (k == GS_EMPTY) return -1;
        s = (s + 1) & H.mask;
    }
    return -1;
}

// ---------------------------------------------------------------- launch helpers (host)
#define GS_CHECK(call)                                                  \
    do {                                                                \
        cudaError_t _e = (call);                                        \
        if (_e != cudaSuccess) return gs_fail_cuda(_e, #call, __FILE__, __LINE__); \
    } while (0)

int gs_fail_cuda(cudaError_t e, const char *what, const char *file, int line);
// process-wide count of this library's kernel launches (for the stats)
void gs_count_launch(void);
long long gs_launch_count(void);
#define GS_LAUNCH(kernel, grid, block, smem, stream) gs_count_launch(), kernel<<<(grid), (block), (smem), (stream)>>>
int gs_fail(int code, const char *fmt, ...);

// device-wide exclusive scan of n int64 values (in place); total -> *d_total (device)
int gs_scan_i64(int64_t *d_vals, int64_t n, int64_t *d_total, cudaStream_t st);
// workspace allocation on the stream-ordered pool
int gs_alloc(void **p, size_t bytes, cudaStream_t st);
void gs_free(void *p, cudaStream_t st);
