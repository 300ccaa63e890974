// gs_bin.cu -- atom preparation and the uniform cell list: per-cell counts
// and their exclusive scan give the cell offsets, and stable radix passes on
// the cell index (gs_radix.cuh) order the atoms by cell, ascending atom index
// within a cell, in time bounded by the number of atoms.  The cell list
// drives the neighbourhood truncation of section 2.2.1: only atoms whose
// cutoff sphere meets a cube (a point) are summed.
#include "gs_host.cuh"
#include "gs_radix.cuh"

// order-preserving map of doubles to unsigned integers (for atomic min/max)
__device__ __forceinline__ unsigned long long dbl_ord(double v)
{
    unsigned long long b = (unsigned long long)__double_as_longlong(v);
    return (b >> 63) ? ~b : (b | 0x8000000000000000ull);
}
__host__ __device__ inline double ord_dbl(unsigned long long o)
{
    unsigned long long b = (o >> 63) ? (o & 0x7fffffffffffffffull) : ~o;
    union { unsigned long long u; double d; } x;
    x.u = b;
    return x.d;
}

// per atom: validate, cutoff radius^2 = r^2 + KD (rounded like r*r then +KD),
// weight exp(D r^2); reduce bounding box and max cutoff^2
__global__ void k_prep(const double *__restrict__ xyz, const double *__restrict__ r, int64_t n, double D, double KD,
                       double *__restrict__ R2, double *__restrict__ w, unsigned long long *__restrict__ red,
                       unsigned *__restrict__ status)
{
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, rmax = 0;
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x) {
        double ri = r[i];
        double x[3] = {xyz[3 * i], xyz[3 * i + 1], xyz[3 * i + 2]};
        bool ok = isfinite(ri) && ri >= 0.0 && isfinite(x[0]) && isfinite(x[1]) && isfinite(x[2]);
        if (!ok) { atomicOr(status, GS_ST_INPUT); continue; }
        double r2 = __dadd_rn(__dmul_rn(ri, ri), KD);
        R2[i] = r2;
        w[i] = exp(__dmul_rn(D, __dmul_rn(ri, ri)));
        rmax = fmax(rmax, r2);
        for (int a = 0; a < 3; a++) { lo[a] = fmin(lo[a], x[a]); hi[a] = fmax(hi[a], x[a]); }
    }
    for (int o = 16; o > 0; o >>= 1) {
        for (int a = 0; a < 3; a++) {
            lo[a] = fmin(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmax(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
        rmax = fmax(rmax, __shfl_xor_sync(0xffffffffu, rmax, o));
    }
    if ((threadIdx.x & 31) == 0) {
        for (int a = 0; a < 3; a++) {
            atomicMin(&red[a], dbl_ord(lo[a]));
            atomicMax(&red[3 + a], dbl_ord(hi[a]));
        }
        atomicMax(&red[6], dbl_ord(rmax));
    }
}

__global__ void k_red_init(unsigned long long *red)
{
    for (int a = 0; a < 3; a++) { red[a] = ~0ull; red[3 + a] = 0ull; }
    red[6] = 0ull;
}

__device__ __forceinline__ int cell_of(double x, double o, double inv, int dim)
{
    double f = floor(__dmul_rn(__dsub_rn(x, o), inv));
    int c = f < 0.0 ? 0 : (f >= (double)dim ? dim - 1 : (int)f);
    return c;
}

__global__ void k_cell_count(const double *__restrict__ xyz, int64_t n, double ox, double oy, double oz,
                             double inv, int cx, int cy, int cz, int32_t *__restrict__ cell_of_atom,
                             int64_t *__restrict__ counts)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int a = cell_of(xyz[3 * i], ox, inv, cx);
    int b = cell_of(xyz[3 * i + 1], oy, inv, cy);
    int c = cell_of(xyz[3 * i + 2], oz, inv, cz);
    int k = a + cx * (b + cy * c);
    cell_of_atom[i] = k;
    atomicAdd((unsigned long long *)&counts[k], 1ull);
}

__global__ void k_cell_starts(const int64_t *__restrict__ start, int64_t ncell, int32_t *__restrict__ cell_start)
{
    int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (k <= ncell) cell_start[k] = (int32_t)start[k];
}

__global__ void k_gather_atoms(const int32_t *__restrict__ perm, int64_t n, const double *__restrict__ xyz,
                               const double *__restrict__ r, const double *__restrict__ R2,
                               const double *__restrict__ w, double ox, double oy, double oz, double cell,
                               int cdx, int cdy, int cdz, double *__restrict__ ax,
                               double *__restrict__ ay, double *__restrict__ az, double *__restrict__ ar,
                               double *__restrict__ aR2, double *__restrict__ aw, float *__restrict__ fx,
                               float *__restrict__ fy, float *__restrict__ fz, float *__restrict__ hx,
                               float *__restrict__ lx, float *__restrict__ hy, float *__restrict__ ly,
                               float *__restrict__ hz, float *__restrict__ lz, float *__restrict__ fw,
                               float *__restrict__ fR2, float *__restrict__ fr2, float *__restrict__ lr2)
{
    int64_t p = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (p >= n) return;
    int64_t i = perm[p];
    double x = xyz[3 * i], y = xyz[3 * i + 1], z = xyz[3 * i + 2];
    ax[p] = x; ay[p] = y; az[p] = z;
    ar[p] = r[i]; aR2[p] = R2[i]; aw[p] = w[i];
    // offsets from the lower corner of the atom's own cell (small, so FP32 keeps ~1e-7 A)
    double inv = 1.0 / cell;
    int cx = cell_of(x, ox, inv, cdx), cy = cell_of(y, oy, inv, cdy), cz = cell_of(z, oz, inv, cdz);
    fx[p] = (float)(x - (ox + cx * cell));
    fy[p] = (float)(y - (oy + cy * cell));
    fz[p] = (float)(z - (oz + cz * cell));
    // centre relative to the origin as hi + lo floats (about 48 bits)
    double rx = x - ox, ry = y - oy, rz = z - oz;
    hx[p] = (float)rx; lx[p] = (float)(rx - (double)hx[p]);
    hy[p] = (float)ry; ly[p] = (float)(ry - (double)hy[p]);
    hz[p] = (float)rz; lz[p] = (float)(rz - (double)hz[p]);
    fw[p] = (float)w[i];
    fR2[p] = (float)R2[i];
    const double rr = r[i] * r[i];
    fr2[p] = (float)rr;
    lr2[p] = (float)(rr - (double)fr2[p]);
}

// ---------------------------------------------------------------- host side

int gs_prep_atoms(const double *d_xyz, const double *d_r, int64_t n, double D, double KD, double *d_R2, double *d_w,
                  double bbox[6], double *r2max, unsigned *d_status, cudaStream_t st)
{
    unsigned long long *red = nullptr;
    int rc = gs_alloc((void **)&red, 7 * sizeof(unsigned long long), st);
    if (rc) return rc;
    GS_LAUNCH(k_red_init, 1, 1, 0, st)(red);
    int blocks = (int)((n + 255) / 256);
    if (blocks > 152 * 8) blocks = 152 * 8;
    if (blocks < 1) blocks = 1;
    GS_LAUNCH(k_prep, blocks, 256, 0, st)(d_xyz, d_r, n, D, KD, d_R2, d_w, red, d_status);
    unsigned long long h[7];
    cudaError_t e = cudaMemcpyAsync(h, red, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = gs_sync(st);
    gs_free(red, st);
    if (e != cudaSuccess) return gs_fail_cuda(e, "prep readback", __FILE__, __LINE__);
    for (int a = 0; a < 6; a++) bbox[a] = ord_dbl(h[a]);
    *r2max = ord_dbl(h[6]);
    return GS_OK;
}

int gs_sort_perm(int32_t *d_keys, int64_t n, int64_t nkeys, int32_t *d_perm, cudaStream_t st)
{
    if (n <= 0) return GS_OK;
    const int passes = rs_passes(nkeys);
    const int64_t nblk = (n + RS_TILE - 1) / RS_TILE;
    int64_t *hist = nullptr;
    int32_t *kb = nullptr, *vb = nullptr;
    int rc = GS_OK;
    if (passes > 0) {
        rc = gs_alloc((void **)&hist, sizeof(int64_t) * (size_t)(256 * nblk + 1), st);
        if (!rc) rc = gs_alloc((void **)&kb, sizeof(int32_t) * (size_t)n, st);
        if (!rc) rc = gs_alloc((void **)&vb, sizeof(int32_t) * (size_t)n, st);
    } else {
        GS_LAUNCH(k_rs_iota, (unsigned)((n + 255) / 256), 256, 0, st)(d_perm, n);
    }
    int32_t *kbuf[2] = {kb, d_keys};
    int32_t *vbuf[2];
    vbuf[(passes - 1) & 1] = d_perm;   // the last pass writes the output
    vbuf[passes & 1] = vb;
    for (int p = 0; p < passes && !rc; p++) {
        const int32_t *kin = p == 0 ? d_keys : kbuf[(p - 1) & 1];
        int32_t *kout = p == passes - 1 ? nullptr : kbuf[p & 1];
        const int32_t *vin = p == 0 ? nullptr : vbuf[(p - 1) & 1];
        GS_LAUNCH(k_rs_hist<int64_t>, (unsigned)nblk, RS_THREADS, 0, st)(kin, n, 8 * p, hist, nblk);
        rc = gs_scan_i64(hist, 256 * nblk, nullptr, st);
        if (!rc)
            GS_LAUNCH(k_rs_scatter<int64_t>, (unsigned)nblk, RS_THREADS, 0, st)(kin, vin, n, 8 * p, hist, nblk, kout,
                                                                              vbuf[p & 1]);
    }
    gs_free(hist, st); gs_free(kb, st); gs_free(vb, st);
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

int gs_build_cells(const double *d_xyz, int64_t n, const double origin[3], double cell, const int cdim[3],
                   int32_t *d_cell_start, int32_t *d_perm, cudaStream_t st)
{
    int64_t ncell = (int64_t)cdim[0] * cdim[1] * cdim[2];
    int64_t *counts = nullptr;
    int32_t *coa = nullptr;
    int rc = gs_alloc((void **)&counts, sizeof(int64_t) * (size_t)(ncell + 1), st);
    if (!rc) rc = gs_alloc((void **)&coa, sizeof(int32_t) * (size_t)n, st);
    if (rc) { gs_free(counts, st); gs_free(coa, st); return rc; }
    cudaMemsetAsync(counts, 0, sizeof(int64_t) * (size_t)(ncell + 1), st);
    double inv = 1.0 / cell;
    unsigned nb = (unsigned)((n + 255) / 256);
    GS_LAUNCH(k_cell_count, nb, 256, 0, st)(d_xyz, n, origin[0], origin[1], origin[2], inv, cdim[0], cdim[1], cdim[2], coa,
                                     counts);
    rc = gs_scan_i64(counts, ncell + 1, nullptr, st);
    if (!rc) GS_LAUNCH(k_cell_starts, (unsigned)((ncell + 1 + 255) / 256), 256, 0, st)(counts, ncell, d_cell_start);
    // atoms grouped by cell, ascending atom index within a cell: stable radix
    // passes on the cell index (time bounded by n whatever the cell sizes)
    if (!rc) rc = gs_sort_perm(coa, n, ncell, d_perm, st);
    gs_free(counts, st); gs_free(coa, st);
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

int gs_gather_atoms(const int32_t *d_perm, int64_t n, const double *d_xyz, const double *d_r, const double *d_R2,
                    const double *d_w, const double origin[3], double cell, const int cdim[3], GsAtomsSoA *soa,
                    cudaStream_t st)
{
    GS_LAUNCH(k_gather_atoms, (unsigned)((n + 255) / 256), 256, 0, st)(d_perm, n, d_xyz, d_r, d_R2, d_w, origin[0],
                                                                 origin[1], origin[2], cell, cdim[0], cdim[1],
                                                                 cdim[2], soa->x, soa->y, soa->z,
                                                                 soa->r, soa->R2, soa->w, soa->fx, soa->fy, soa->fz,
                                                                 soa->hx, soa->lx, soa->hy, soa->ly, soa->hz, soa->lz,
                                                                 soa->fw, soa->fR2, soa->fr2, soa->lr2);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}
