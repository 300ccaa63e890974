// gs_field.cu -- phi and grad phi at points (eq Gaussian1 with the
// neighbourhood truncation of section 2.2.1).  The points are the lattice
// vertices of the accepted cubes (the values the trilinear interpolant of
// eq linear1 takes at the cube corners) or caller-given positions.
//
// One thread per point; candidate atoms come from the cell rows around the
// point, in cell order (ascending atom index inside each cell).  The FP64
// form sums exp(-D (d^2 - r^2)) directly.  The FP32 form takes each atom's
// offset from its cell corner (FP32) and the point's offset from the same
// corner (formed in FP64 once per cell), evaluates the exponential with
// exp2f, sums with Kahan compensation and returns an error bound per point.
#include "gs_host.cuh"

__device__ __forceinline__ void point_of(const GsProblem &P, const uint64_t *vkeys, const double *pts, int64_t i,
                                         double *p)
{
    if (vkeys) {
        uint64_t k = vkeys[i];
        p[0] = gs_lat(P, 0, gk_x(k), P.max_depth);
        p[1] = gs_lat(P, 1, gk_y(k), P.max_depth);
        p[2] = gs_lat(P, 2, gk_z(k), P.max_depth);
    } else {
        p[0] = pts[3 * i]; p[1] = pts[3 * i + 1]; p[2] = pts[3 * i + 2];
    }
}

// cells around point p within the largest cutoff radius; body(begin, end, cx, cy, cz)
template <typename F>
__device__ __forceinline__ void for_point_cells(const GsProblem &P, const double *p, F body)
{
    int c0[3], c1[3];
    for (int a = 0; a < 3; a++) {
        double f0 = floor((p[a] - P.pad - P.origin[a]) * P.inv_cell);
        double f1 = floor((p[a] + P.pad - P.origin[a]) * P.inv_cell);
        c0[a] = f0 < 0 ? 0 : (f0 >= P.cdim[a] ? P.cdim[a] - 1 : (int)f0);
        c1[a] = f1 < 0 ? 0 : (f1 >= P.cdim[a] ? P.cdim[a] - 1 : (int)f1);
    }
    double pad2 = P.pad * P.pad;
    for (int cz = c0[2]; cz <= c1[2]; cz++) {
        double zlo = P.origin[2] + cz * P.cell;
        double gz = fmax(0.0, fmax(zlo - p[2], p[2] - (zlo + P.cell)));
        for (int cy = c0[1]; cy <= c1[1]; cy++) {
            double ylo = P.origin[1] + cy * P.cell;
            double gy = fmax(0.0, fmax(ylo - p[1], p[1] - (ylo + P.cell)));
            double rem2 = pad2 - gy * gy - gz * gz;
            if (rem2 < 0) continue;
            double rem = sqrt(rem2) * (1.0 + 1e-12) + 1e-12;
            double f0 = floor((p[0] - rem - P.origin[0]) * P.inv_cell);
            double f1 = floor((p[0] + rem - P.origin[0]) * P.inv_cell);
            int x0 = f0 < c0[0] ? c0[0] : (int)f0;
            int x1 = f1 > c1[0] ? c1[0] : (int)f1;
            int64_t row = (int64_t)P.cdim[0] * (cy + (int64_t)P.cdim[1] * cz);
            for (int cx = x0; cx <= x1; cx++) body(P.cell_start[row + cx], P.cell_start[row + cx + 1], cx, cy, cz);
        }
    }
}

__global__ void __launch_bounds__(128) k_field_f64(GsProblem P, const uint64_t *vkeys, const double *pts, int64_t n,
                                                   double *__restrict__ phi, double *__restrict__ grad,
                                                   unsigned long long *terms)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long cnt = 0;
    if (i < n) {
        double p[3];
        point_of(P, vkeys, pts, i, p);
        double s = 0, g0 = 0, g1 = 0, g2 = 0;
        const double m2D = -2.0 * P.D;
        for_point_cells(P, p, [&](int b, int e, int, int, int) {
            for (int k = b; k < e; k++) {
                double dx = __dsub_rn(p[0], P.ax[k]), dy = __dsub_rn(p[1], P.ay[k]), dz = __dsub_rn(p[2], P.az[k]);
                double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                if (d2 > P.aR2[k]) continue;
                double r = P.ar[k];
                double t = exp(-P.D * (d2 - r * r));
                s += t;
                g0 = fma(m2D * dx, t, g0);
                g1 = fma(m2D * dy, t, g1);
                g2 = fma(m2D * dz, t, g2);
                cnt++;
            }
        });
        phi[i] = s;
        if (grad) { grad[3 * i] = g0; grad[3 * i + 1] = g1; grad[3 * i + 2] = g2; }
    }
    if (terms) {
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(terms, cnt);
    }
}

// FP32 form with per-point error bound err = sum of |term| * eps_term + Kahan residual bound
__global__ void __launch_bounds__(128) k_field_f32(GsProblem P, const uint64_t *vkeys, const double *pts, int64_t n,
                                                   double *__restrict__ phi, double *__restrict__ grad,
                                                   float *__restrict__ err, unsigned long long *terms)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long cnt = 0;
    if (i < n) {
        double p[3];
        point_of(P, vkeys, pts, i, p);
        float s = 0.f, comp = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, absum = 0.f;
        const float nDl2e = (float)(-P.D * 1.4426950408889634);
        const float m2D = (float)(-2.0 * P.D);
        for_point_cells(P, p, [&](int b, int e, int cx, int cy, int cz) {
            // point offset from this cell's lower corner, formed in FP64
            float qx = (float)(p[0] - (P.origin[0] + cx * P.cell));
            float qy = (float)(p[1] - (P.origin[1] + cy * P.cell));
            float qz = (float)(p[2] - (P.origin[2] + cz * P.cell));
            for (int k = b; k < e; k++) {
                float dx = qx - P.fx[k], dy = qy - P.fy[k], dz = qz - P.fz[k];
                float d2 = dx * dx + dy * dy + dz * dz;
                float r = (float)P.ar[k];
                // same membership as FP64 except within rounding of the boundary,
                // where terms are ~cutoff_rel*c and inside the error bound
                if (d2 > (float)P.aR2[k]) continue;
                float t = exp2f(nDl2e * (d2 - r * r));
                float y = t - comp;
                float u = s + y;
                comp = (u - s) - y;
                s = u;
                absum += t;
                g0 = fmaf(m2D * dx, t, g0);
                g1 = fmaf(m2D * dy, t, g1);
                g2 = fmaf(m2D * dz, t, g2);
                cnt++;
            }
        });
        phi[i] = (double)s - (double)comp;
        if (grad) { grad[3 * i] = g0; grad[3 * i + 1] = g1; grad[3 * i + 2] = g2; }
        // per-term relative error: exp2f (2 ulp) + argument rounding: the
        // argument D(d^2 - r^2) carries ~4 ulp of d^2 (<= 40 A^2) times D
        // -> about 1e-5 * t absolute on the largest terms, 3e-6 typical
        if (err) err[i] = 2e-5f * absum + 1e-7f * (float)P.c;
    }
    if (terms) {
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(terms, cnt);
    }
}

int gs_field_f64(const GsProblem &P, const uint64_t *d_vkeys, const double *d_points, int64_t n, double *d_phi,
                 double *d_grad, unsigned long long *d_terms, cudaStream_t st)
{
    if (n <= 0) return GS_OK;
    GS_LAUNCH(k_field_f64, (unsigned)((n + 127) / 128), 128, 0, st)(P, d_vkeys, d_points, n, d_phi, d_grad, d_terms);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

int gs_field_f32(const GsProblem &P, const uint64_t *d_vkeys, const double *d_points, int64_t n, double *d_phi,
                 double *d_grad, float *d_err, unsigned long long *d_terms, cudaStream_t st)
{
    if (n <= 0) return GS_OK;
    GS_LAUNCH(k_field_f32, (unsigned)((n + 127) / 128), 128, 0, st)(P, d_vkeys, d_points, n, d_phi, d_grad, d_err, d_terms);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// ---------------------------------------------------------------- mixed field
// FP32 values everywhere, FP64 re-evaluation of the vertices whose sign
// relative to c (the inside test of the triangulation) is within the FP32
// error bound.
__global__ void k_field_flag(const double *phi, const float *err, int64_t n, double c, int64_t *cnt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    cnt[i] = fabs(phi[i] - c) <= 4.0 * (double)err[i] ? 1 : 0;
}
__global__ void k_field_gather(const int64_t *off, int64_t n, const uint64_t *vkeys, uint64_t *sub_keys, int64_t *sub_idx)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n || off[i + 1] == off[i]) return;
    sub_keys[off[i]] = vkeys[i];
    sub_idx[off[i]] = i;
}
__global__ void k_field_scatter(const double *sub_phi, const int64_t *sub_idx, int64_t m, double *phi)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) phi[sub_idx[t]] = sub_phi[t];
}

int gs_field_mixed(const GsProblem &P, const uint64_t *d_vkeys, int64_t n, double *d_phi, unsigned long long *d_terms,
                   int64_t *n_rechecked, cudaStream_t st)
{
    *n_rechecked = 0;
    if (n <= 0) return GS_OK;
    float *err = nullptr;
    int64_t *cnt = nullptr, *tot = nullptr;
    int rc = gs_alloc((void **)&err, sizeof(float) * (size_t)n, st);
    if (!rc) rc = gs_alloc((void **)&cnt, sizeof(int64_t) * (size_t)(n + 1), st);
    if (!rc) rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
    if (!rc) rc = gs_field_f32(P, d_vkeys, nullptr, n, d_phi, nullptr, err, d_terms, st);
    if (!rc) {
        cudaMemsetAsync(cnt + n, 0, sizeof(int64_t), st);
        GS_LAUNCH(k_field_flag, (unsigned)((n + 255) / 256), 256, 0, st)(d_phi, err, n, P.c, cnt);
        rc = gs_scan_i64(cnt, n + 1, tot, st);
    }
    int64_t m = 0;
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(&m, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = gs_fail_cuda(e, "field recheck count", __FILE__, __LINE__);
    }
    if (!rc && m > 0) {
        uint64_t *sk = nullptr;
        int64_t *si = nullptr;
        double *sp = nullptr;
        rc = gs_alloc((void **)&sk, sizeof(uint64_t) * (size_t)m, st);
        if (!rc) rc = gs_alloc((void **)&si, sizeof(int64_t) * (size_t)m, st);
        if (!rc) rc = gs_alloc((void **)&sp, sizeof(double) * (size_t)m, st);
        if (!rc) {
            GS_LAUNCH(k_field_gather, (unsigned)((n + 255) / 256), 256, 0, st)(cnt, n, d_vkeys, sk, si);
            rc = gs_field_f64(P, sk, nullptr, m, sp, nullptr, nullptr, st);
        }
        if (!rc) GS_LAUNCH(k_field_scatter, (unsigned)((m + 255) / 256), 256, 0, st)(sp, si, m, d_phi);
        gs_free(sk, st); gs_free(si, st); gs_free(sp, st);
    }
    gs_free(err, st); gs_free(cnt, st); gs_free(tot, st);
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    *n_rechecked = m;
    return GS_OK;
}
