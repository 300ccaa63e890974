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
// gs_ex2, sums with Kahan compensation and returns an error bound per point.
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

// the warp box filter of the warp-cooperative field kernels: an atom is
// staged only if its cutoff sphere reaches the box of the warp's vertices.
// The box and the centre are hi parts of offsets from the origin (each
// within 6e-8 |x| of the exact offset) and the gaps round once more, so each
// gap is lowered by 1e-3 A + 4e-7 |x| and the sphere grown by 1% + 0.01 A^2:
// every atom that some vertex of the warp accepts passes
__device__ __forceinline__ bool dw_box_reaches(const float *lo, const float *hi, float x, float y, float z, float R2)
{
    const float gx = fmaxf(0.f, fmaxf(lo[0] - x, x - hi[0]) - fmaf(4e-7f, fabsf(x), 1e-3f));
    const float gy = fmaxf(0.f, fmaxf(lo[1] - y, y - hi[1]) - fmaf(4e-7f, fabsf(y), 1e-3f));
    const float gz = fmaxf(0.f, fmaxf(lo[2] - z, z - hi[2]) - fmaf(4e-7f, fabsf(z), 1e-3f));
    return gx * gx + gy * gy + gz * gz <= fmaf(R2, 1.01f, 0.01f);
}

// FP64 field.  Candidates are screened with the FP32 distance (two-float
// offsets from the origin) and a relative margin; inside the margin the
// membership is the exact FP64 test.  t = w exp(-D d^2) with w = exp(D r^2).
template <bool GRAD>
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
        const double m2D = -2.0 * P.D, nD = -P.D;
        float ph[3], pl[3];
        for (int a = 0; a < 3; a++) {
            double rel = p[a] - P.origin[a];
            ph[a] = (float)rel;
            pl[a] = (float)(rel - (double)ph[a]);
        }
        gs_for_rows(P, ph, ph, [&](int b, int e, int64_t, int) {
            for (int k = b; k < e; k++) {
                float fx = (ph[0] - P.hx[k]) + (pl[0] - P.lx[k]);
                float fy = (ph[1] - P.hy[k]) + (pl[1] - P.ly[k]);
                float fz = (ph[2] - P.hz[k]) + (pl[2] - P.lz[k]);
                float f2 = fx * fx + fy * fy + fz * fz;
                const float R2 = P.fR2[k];
                if (f2 > R2 * (1.f + 1e-5f) + 1e-5f) continue;
                double dx = __dsub_rn(p[0], P.ax[k]), dy = __dsub_rn(p[1], P.ay[k]), dz = __dsub_rn(p[2], P.az[k]);
                double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                if (d2 > P.aR2[k]) continue;
                double t = P.aw[k] * gs_exp(nD * d2);
                s += t;
                if (GRAD) {
                    g0 = fma(m2D * dx, t, g0);
                    g1 = fma(m2D * dy, t, g1);
                    g2 = fma(m2D * dz, t, g2);
                }
                cnt++;
            }
        });
        phi[i] = s;
        if (GRAD) { grad[3 * i] = g0; grad[3 * i + 1] = g1; grad[3 * i + 2] = g2; }
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
        float s = 0.f, comp = 0.f, g0 = 0.f, g1 = 0.f, g2 = 0.f, eacc = 0.f;
        const float nDl2e = (float)(-P.D * 1.4426950408889634);
        const float Df = (float)P.D;
        const float m2D = (float)(-2.0 * P.D);
        // the point relative to the origin as hi + lo floats
        float ph[3], pl[3];
        for (int a = 0; a < 3; a++) {
            double rel = p[a] - P.origin[a];
            ph[a] = (float)rel;
            pl[a] = (float)(rel - (double)ph[a]);
        }
        gs_for_rows(P, ph, ph, [&](int b, int e, int64_t, int) {
            for (int k = b; k < e; k++) {
                float dx = (ph[0] - P.hx[k]) + (pl[0] - P.lx[k]);
                float dy = (ph[1] - P.hy[k]) + (pl[1] - P.ly[k]);
                float dz = (ph[2] - P.hz[k]) + (pl[2] - P.lz[k]);
                float d2 = dx * dx + dy * dy + dz * dz;
                // membership as in FP64 except within rounding of the cutoff
                // sphere, where a term is ~cutoff_rel * c and inside the bound
                if (d2 > P.fR2[k]) continue;
                float r2 = P.fr2[k];
                float t = gs_ex2(nDl2e * (d2 - r2));
                float y = t - comp;
                float u = s + y;
                comp = (u - s) - y;
                s = u;
                // this term's error: ex2 (2 ulp) and the rounding of its
                // argument, about 3 ulp of d^2 and r^2 times D
                eacc = fmaf(t, 3e-7f + 3e-7f * Df * (d2 + r2), eacc);
                g0 = fmaf(m2D * dx, t, g0);
                g1 = fmaf(m2D * dy, t, g1);
                g2 = fmaf(m2D * dz, t, g2);
                cnt++;
            }
        });
        phi[i] = (double)s - (double)comp;
        if (grad) { grad[3 * i] = g0; grad[3 * i + 1] = g1; grad[3 * i + 2] = g2; }
        // bound per point: the terms' own errors, the compensated sum's
        // residual, and the few terms at the cutoff sphere (each ~cutoff_rel*c)
        // that the FP32 membership test may include or drop
        if (err) err[i] = eacc + 2.4e-7f * s + 4e-8f * (float)P.c;
    }
    if (terms) {
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(terms, cnt);
    }
}

// FP32 field at lattice vertices, warp-cooperative: a warp takes 32
// consecutive vertices (neighbours on the lattice: the vertex order follows
// the cube order), walks the cell rows of their bounding box once, and
// stages 32 candidate atoms at a time in shared memory (offsets from the
// origin as hi + lo floats, cutoff^2, r^2); every lane then sums over the
// staged atoms from broadcast reads.  Rows come in the order of the
// per-vertex walk and each row's range covers the vertex's own, so each
// vertex sums the same terms in the same order, with the same membership
// test and error bound as k_field_f32.
//
// Tile shape (template): WARPS warps per block, VPL vertices per lane (a
// warp tile of 32 VPL consecutive vertices; lane l holds vertices l, l + 32,
// ...).  A larger tile stages each candidate for more vertices but widens
// the bounding box; the sums are the same for every shape (each vertex sees
// its own atoms in the same order), so the shape is free to be tuned.
template <int WARPS, int VPL>
__global__ void __launch_bounds__(32 * WARPS) k_field_f32w(GsProblem P, const uint64_t *__restrict__ vkeys, int64_t n,
                                                           double *__restrict__ phi, float *__restrict__ err,
                                                           unsigned long long *terms)
{
    __shared__ float4 s_a[WARPS][32];   // hx, hy, hz, fR2
    __shared__ float4 s_b[WARPS][32];   // lx, ly, lz, fr2
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int64_t i0 = ((int64_t)blockIdx.x * WARPS + w) * (32 * VPL) + lane;
    bool valid[VPL];
    float ph[VPL][3], pl[VPL][3];
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
#pragma unroll
    for (int v = 0; v < VPL; v++) {
        const int64_t i = i0 + 32 * v;
        valid[v] = i < n;
        for (int a = 0; a < 3; a++) ph[v][a] = pl[v][a] = 0.f;
        if (valid[v]) {
            double p[3];
            point_of(P, vkeys, nullptr, i, p);
            for (int a = 0; a < 3; a++) {
                double rel = p[a] - P.origin[a];
                ph[v][a] = (float)rel;
                pl[v][a] = (float)(rel - (double)ph[v][a]);
                lo[a] = fminf(lo[a], ph[v][a]);
                hi[a] = fmaxf(hi[a], ph[v][a]);
            }
        }
    }
    // the warp's bounding box
    for (int a = 0; a < 3; a++)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(0xffffffffu, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(0xffffffffu, hi[a], o));
        }
    if (!(lo[0] <= hi[0])) return;   // no vertex in this warp (uniform)
    const float nDl2e = (float)(-P.D * 1.4426950408889634);
    const float Df = (float)P.D;
    float s[VPL], comp[VPL], eacc[VPL];
#pragma unroll
    for (int v = 0; v < VPL; v++) s[v] = comp[v] = eacc[v] = 0.f;
    unsigned long long cnt = 0;
    const unsigned below = (1u << lane) - 1u;
    gs_warp_candidates(P, lo, hi, lane, [&](int k) {
        float4 A = make_float4(0.f, 0.f, 0.f, 0.f);
        bool keep = false;
        if (k >= 0) {
            A = make_float4(P.hx[k], P.hy[k], P.hz[k], P.fR2[k]);
            keep = dw_box_reaches(lo, hi, A.x, A.y, A.z, A.w);
        }
        const unsigned have = __ballot_sync(0xffffffffu, keep);
        if (keep) {
            const int slot = __popc(have & below);
            s_a[w][slot] = A;
            s_b[w][slot] = make_float4(P.lx[k], P.ly[k], P.lz[k], P.fr2[k]);
        }
        __syncwarp();
        const int m = __popc(have);
#pragma unroll
        for (int v = 0; v < VPL; v++) {
            if (!valid[v]) continue;
            for (int j = 0; j < m; j++) {
                const float4 a = s_a[w][j], b = s_b[w][j];
                const float dx = (ph[v][0] - a.x) + (pl[v][0] - b.x);
                const float dy = (ph[v][1] - a.y) + (pl[v][1] - b.y);
                const float dz = (ph[v][2] - a.z) + (pl[v][2] - b.z);
                const float d2 = dx * dx + dy * dy + dz * dz;
                if (d2 > a.w) continue;
                const float t = gs_ex2(nDl2e * (d2 - b.w));
                const float y = t - comp[v];
                const float u = s[v] + y;
                comp[v] = (u - s[v]) - y;
                s[v] = u;
                eacc[v] = fmaf(t, 3e-7f + 3e-7f * Df * (d2 + b.w), eacc[v]);
                cnt++;
            }
        }
        __syncwarp();
    });
#pragma unroll
    for (int v = 0; v < VPL; v++) {
        if (!valid[v]) continue;
        const int64_t i = i0 + 32 * v;
        phi[i] = (double)s[v] - (double)comp[v];
        if (err) err[i] = eacc[v] + 2.4e-7f * s[v] + 4e-8f * (float)P.c;
    }
    if (terms) {
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
        if (lane == 0 && cnt) atomicAdd(terms, cnt);
    }
}

// the tile shapes the tuner chooses from: (warps per block, vertices per lane)
static const int FW_SHAPES[][2] = {{8, 1}, {4, 1}, {8, 2}, {4, 2}};
#define FW_NSHAPES 4

static void launch_field_f32w(int shape, const GsProblem &P, const uint64_t *d_vkeys, int64_t n, double *d_phi,
                              float *d_err, unsigned long long *d_terms, cudaStream_t st)
{
    const int W = FW_SHAPES[shape][0], V = FW_SHAPES[shape][1];
    const unsigned grid = (unsigned)((n + 32 * W * V - 1) / (32 * W * V));
    switch (shape) {
    case 0: GS_LAUNCH((k_field_f32w<8, 1>), grid, 256, 0, st)(P, d_vkeys, n, d_phi, d_err, d_terms); break;
    case 1: GS_LAUNCH((k_field_f32w<4, 1>), grid, 128, 0, st)(P, d_vkeys, n, d_phi, d_err, d_terms); break;
    case 2: GS_LAUNCH((k_field_f32w<8, 2>), grid, 256, 0, st)(P, d_vkeys, n, d_phi, d_err, d_terms); break;
    default: GS_LAUNCH((k_field_f32w<4, 2>), grid, 128, 0, st)(P, d_vkeys, n, d_phi, d_err, d_terms); break;
    }
}

int gs_field_f64(const GsProblem &P, const uint64_t *d_vkeys, const double *d_points, int64_t n, double *d_phi,
                 double *d_grad, unsigned long long *d_terms, cudaStream_t st)
{
    if (n <= 0) return GS_OK;
    if (d_grad)
        GS_LAUNCH(k_field_f64<true>, (unsigned)((n + 127) / 128), 128, 0, st)(P, d_vkeys, d_points, n, d_phi, d_grad,
                                                                             d_terms);
    else
        GS_LAUNCH(k_field_f64<false>, (unsigned)((n + 127) / 128), 128, 0, st)(P, d_vkeys, d_points, n, d_phi, d_grad,
                                                                              d_terms);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

int gs_field_f32(const GsProblem &P, const uint64_t *d_vkeys, const double *d_points, int64_t n, double *d_phi,
                 double *d_grad, float *d_err, unsigned long long *d_terms, cudaStream_t st)
{
    if (n <= 0) return GS_OK;
    if (d_vkeys && !d_grad) {   // lattice vertices: the warp-cooperative form, tile shape tuned
        int rc = gs_tune_run("k_field_f32w", n, FW_NSHAPES, st, [&](int shape, unsigned long long *scratch) {
            launch_field_f32w(shape, P, d_vkeys, n, d_phi, d_err, scratch ? (d_terms ? scratch : nullptr) : d_terms,
                              st);
        });
        if (rc) return rc;
    } else
        GS_LAUNCH(k_field_f32, (unsigned)((n + 127) / 128), 128, 0, st)(P, d_vkeys, d_points, n, d_phi, d_grad, d_err,
                                                                       d_terms);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// ---------------------------------------------------------------- double-word re-evaluation
// The mixed form's second opinion on a lattice vertex whose FP32 bound is
// too wide: phi in double-word FP32 arithmetic, each value an unevaluated
// sum hi + lo of two floats.  The rounding error of one addition is exact
// by TwoSum (Knuth) or FastTwoSum (Dekker, |a| >= |b|), that of a product
// by TwoProduct with an FMA; the explicit __fadd_rn / __fmul_rn / __fmaf_rn
// keep the compiler from contracting them.  It runs on the FP32 pipes (GB300
// issues FP64 at 1/64 of their rate) and returns phi with a bound near
// 5e-10 relative (offsets of 600 A), some 2000 times tighter than the FP32
// sum's.
//
// One term t = exp(-D (d^2 - r^2)) = 2^y with y = K (r^2 - d^2), K = D log2(e):
//   d^2    from the two-float offsets: per axis s + e = ph - ah exactly,
//          lo = e + (pl - al), dx^2 = s^2 (TwoProduct) + (2 s + lo) lo; the
//          three s^2 summed by TwoSum;
//   y      (r^2 - d^2) by TwoSum with r^2 = fr2 + lr2, times K = Kh + Kl;
//   2^y    = 2^n 2^(j/64) e^(g ln 2), n = rint(y), j = rint(64 (y - n)),
//          |g| <= 1/128; 2^(j/64) from a double-word table; e^s = 1 + s + Q
//          with Q = s^2 (1/2 + s/6 + s^2/24 + s^3/120) in FP32 (|s| < 0.0055:
//          Q < 1.5e-5, so its FP32 error is below 1e-11 of the term, and the
//          truncation below 4e-17);
//   sum    double-word, renormalised after each term.
// Error bound per term (relative; u = 2^-24, L the largest vertex offset
// from the origin, R the largest cutoff radius, |dx| <= R):
//   the offsets: the hi + lo floats are within u^2 |x| of the FP64 offsets,
//   and the lo parts (up to 2.1 u (L + R)) round twice more, so each axis
//   offset is off by at most delta = u^2 (6.2 L + 4.1 R), d^2 by 2 sqrt(3) R
//   delta from that; forming d^2 rounds the (2 s + lo) lo parts and their
//   sum (six roundings of values up to 2 sqrt(3) R 2.1 u (L + R) + u R^2),
//   r^2 - d^2 two more, y = K z eight u^2 K R^2: together y is off by at most
//   K u^2 (85 R L + 113 R^2), and t by ln 2 times that (ln 2 K = D);
//   the exponential stage adds at most 2e-11 (Q, the table's lo parts and
//   four roundings of lo parts, each below 4e-12);
//   the sum of m positive terms adds u^2 (3 m + 2) S, the final hi + lo in
//   FP64 2^-53 S.
// So err = S (D u^2 (90 R L + 120 R^2) + 2e-11 + u^2 (3 m + 2) + 2^-52),
// inflated by 1% for its own rounding.  Membership is the FP64 field's: the
// FP32 distance screens with a 1e-5 relative margin and inside the margin
// the exact FP64 test decides.
__constant__ float2 c_dw_exp2[65];   // 2^(j/64), j = -32..32, as (hi, lo)

struct DWf { float h, l; };
__device__ __forceinline__ DWf dw_two_sum(float a, float b)
{
    const float s = __fadd_rn(a, b), bb = __fsub_rn(s, a);
    return {s, __fadd_rn(__fsub_rn(a, __fsub_rn(s, bb)), __fsub_rn(b, bb))};
}
__device__ __forceinline__ DWf dw_fast_two_sum(float a, float b)   // |a| >= |b|
{
    const float s = __fadd_rn(a, b);
    return {s, __fsub_rn(b, __fsub_rn(s, a))};
}
__device__ __forceinline__ DWf dw_two_prod(float a, float b)
{
    const float p = __fmul_rn(a, b);
    return {p, __fmaf_rn(a, b, -p)};
}

// constants of one double-word evaluation
struct DwConst {
    float Kh, Kl;     // D log2(e)
    float L2h, L2l;   // ln 2
};

// add atom k's term to the double-word sum (Sh, Sl) of the point (p in FP64;
// ph + pl its offset from the origin); ah + al the atom's offset, R2 its
// cutoff^2 (FP32), r2h + r2l its r^2
__device__ __forceinline__ void dw_add_atom(const GsProblem &P, const double *p, const float *ph, const float *pl,
                                            const float *ah, const float *al, float R2, float r2h, float r2l, int k,
                                            const DwConst &C, const float2 *tab, float &Sh, float &Sl, int &m)
{
    const DWf sx = dw_two_sum(ph[0], -ah[0]), sy = dw_two_sum(ph[1], -ah[1]), sz = dw_two_sum(ph[2], -ah[2]);
    const float ox = __fsub_rn(pl[0], al[0]), oy = __fsub_rn(pl[1], al[1]), oz = __fsub_rn(pl[2], al[2]);
    // the FP32 screen (the FP64 field's prefilter)
    const float fx = sx.h + ox, fy = sy.h + oy, fz = sz.h + oz;
    const float f2 = fx * fx + fy * fy + fz * fz;
    if (f2 > R2 * (1.f + 1e-5f) + 1e-5f) return;
    if (f2 >= R2 * (1.f - 1e-5f) - 1e-5f) {
        // near the cutoff sphere: the exact FP64 membership test
        const double dx = __dsub_rn(p[0], P.ax[k]), dy = __dsub_rn(p[1], P.ay[k]), dz = __dsub_rn(p[2], P.az[k]);
        const double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
        if (d2 > P.aR2[k]) return;
    }
    // d^2 = sum over axes of s^2 + (2 s + lo) lo, lo = e + (pl - al)
    const float lx = __fadd_rn(sx.l, ox), ly = __fadd_rn(sy.l, oy), lz = __fadd_rn(sz.l, oz);
    const DWf px = dw_two_prod(sx.h, sx.h), py = dw_two_prod(sy.h, sy.h), pz = dw_two_prod(sz.h, sz.h);
    const float qx = __fmaf_rn(__fadd_rn(__fadd_rn(sx.h, sx.h), lx), lx, px.l);
    const float qy = __fmaf_rn(__fadd_rn(__fadd_rn(sy.h, sy.h), ly), ly, py.l);
    const float qz = __fmaf_rn(__fadd_rn(__fadd_rn(sz.h, sz.h), lz), lz, pz.l);
    const DWf u1 = dw_two_sum(px.h, py.h), u2 = dw_two_sum(u1.h, pz.h);
    const float d2l = __fadd_rn(__fadd_rn(u1.l, u2.l), __fadd_rn(__fadd_rn(qx, qy), qz));
    // z = r^2 - d^2, y = K z
    const DWf z = dw_two_sum(r2h, -u2.h);
    const float zl = __fadd_rn(z.l, __fsub_rn(r2l, d2l));
    const float yh = __fmul_rn(C.Kh, z.h);
    const float yl = __fmaf_rn(C.Kh, zl, __fmaf_rn(C.Kl, z.h, __fmaf_rn(C.Kh, z.h, -yh)));
    // 2^y = 2^nn 2^(jj/64) e^((g + yl) ln 2); yh - nn and f - jj/64 are exact.
    // The mixed form's range check (D R^2 <= 80) keeps |y| below 116; the
    // clamps only keep the table index and the exponent field in range for
    // any input (a non-finite point, say)
    const float nn = fminf(fmaxf(rintf(yh), -120.f), 120.f);
    const float f = __fsub_rn(yh, nn);
    const float jj = rintf(__fmul_rn(f, 64.f));
    const DWf r = dw_two_sum(__fsub_rn(f, __fmul_rn(jj, 0.015625f)), yl);
    const float sh = __fmul_rn(C.L2h, r.h);
    const float sl = __fmaf_rn(C.L2h, r.l, __fmaf_rn(C.L2l, r.h, __fmaf_rn(C.L2h, r.h, -sh)));
    const float q = __fmaf_rn(sh, __fmaf_rn(sh, __fmaf_rn(sh, 1.f / 120.f, 1.f / 24.f), 1.f / 6.f), 0.5f);
    const float Q = __fmaf_rn(sh, sl, __fmul_rn(__fmul_rn(sh, sh), q));
    const DWf E = dw_fast_two_sum(1.f, sh);
    const float el = __fadd_rn(E.l, __fadd_rn(sl, Q));
    const float2 T = tab[min(max((int)jj, -32), 32) + 32];
    const DWf TE = dw_two_prod(T.x, E.h);
    const float tl0 = __fmaf_rn(T.x, el, __fmaf_rn(T.y, E.h, TE.l));
    const float sc = __int_as_float(((int)nn + 127) << 23);
    const float th = __fmul_rn(TE.h, sc), tl = __fmul_rn(tl0, sc);
    const DWf U = dw_two_sum(Sh, th);
    const DWf V = dw_fast_two_sum(U.h, __fadd_rn(Sl, __fadd_rn(tl, U.l)));
    Sh = V.h;
    Sl = V.l;
    m++;
}

// A warp takes 32 consecutive points.  When their box is compact it walks
// the box's cell rows once and stages 32 candidates at a time in shared
// memory (the warp box filter drops the atoms that reach no point of the
// box); when the points are spread out (a sparse selection of the lattice)
// each lane walks the rows around its own point.  Either way a point sums
// its own atoms in cell-row order.
template <int WARPS>
__global__ void __launch_bounds__(32 * WARPS) k_field_dw(GsProblem P, const uint64_t *__restrict__ vkeys,
                                                         const double *__restrict__ pts, int64_t n, DwConst C,
                                                         double *__restrict__ phi, float *__restrict__ err,
                                                         unsigned long long *terms)
{
    __shared__ float4 s_a[WARPS][32];   // hx, hy, hz, fR2
    __shared__ float4 s_b[WARPS][32];   // lx, ly, lz, fr2
    __shared__ float2 s_c[WARPS][32];   // lr2, atom index (bits)
    __shared__ float2 s_t[65];
    for (int k = threadIdx.x; k < 65; k += blockDim.x) s_t[k] = c_dw_exp2[k];
    __syncthreads();
    const unsigned full = 0xffffffffu;
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const int64_t i = ((int64_t)blockIdx.x * WARPS + w) * 32 + lane;
    const bool valid = i < n;
    double p[3] = {0.0, 0.0, 0.0};
    float ph[3] = {0.f, 0.f, 0.f}, pl[3] = {0.f, 0.f, 0.f};
    float lo[3] = {INFINITY, INFINITY, INFINITY}, hi[3] = {-INFINITY, -INFINITY, -INFINITY};
    if (valid) {
        point_of(P, vkeys, pts, i, p);
        for (int a = 0; a < 3; a++) {
            const double rel = p[a] - P.origin[a];
            ph[a] = (float)rel;
            pl[a] = (float)(rel - (double)ph[a]);
            lo[a] = hi[a] = ph[a];
        }
    }
    for (int a = 0; a < 3; a++)
        for (int o = 16; o > 0; o >>= 1) {
            lo[a] = fminf(lo[a], __shfl_xor_sync(full, lo[a], o));
            hi[a] = fmaxf(hi[a], __shfl_xor_sync(full, hi[a], o));
        }
    if (!(lo[0] <= hi[0])) return;   // no point in this warp (uniform)
    float Sh = 0.f, Sl = 0.f;
    int m = 0;
    const float spread = fmaxf(hi[0] - lo[0], fmaxf(hi[1] - lo[1], hi[2] - lo[2]));
    if (spread <= 2.f * P.cell_f) {
        gs_warp_candidates(P, lo, hi, lane, [&](int k) {
            float4 A = make_float4(0.f, 0.f, 0.f, 0.f);
            bool keep = false;
            if (k >= 0) {
                A = make_float4(P.hx[k], P.hy[k], P.hz[k], P.fR2[k]);
                keep = dw_box_reaches(lo, hi, A.x, A.y, A.z, A.w);
            }
            const unsigned kb = __ballot_sync(full, keep);
            if (keep) {
                const int slot = __popc(kb & below);
                s_a[w][slot] = A;
                s_b[w][slot] = make_float4(P.lx[k], P.ly[k], P.lz[k], P.fr2[k]);
                s_c[w][slot] = make_float2(P.lr2[k], __int_as_float(k));
            }
            __syncwarp();
            const int nk = __popc(kb);
            for (int j = 0; valid && j < nk; j++) {
                const float4 a = s_a[w][j], b = s_b[w][j];
                const float2 cc = s_c[w][j];
                const float ah[3] = {a.x, a.y, a.z}, al[3] = {b.x, b.y, b.z};
                dw_add_atom(P, p, ph, pl, ah, al, a.w, b.w, cc.x, __float_as_int(cc.y), C, s_t, Sh, Sl, m);
            }
            __syncwarp();
        });
    } else if (valid) {
        gs_for_rows(P, ph, ph, [&](int b, int e, int64_t, int) {
            for (int k = b; k < e; k++) {
                const float ah[3] = {P.hx[k], P.hy[k], P.hz[k]}, al[3] = {P.lx[k], P.ly[k], P.lz[k]};
                dw_add_atom(P, p, ph, pl, ah, al, P.fR2[k], P.fr2[k], P.lr2[k], k, C, s_t, Sh, Sl, m);
            }
        });
    }
    if (valid) {
        const double S = (double)Sh + (double)Sl;
        phi[i] = S;
        if (err) {
            const double u2 = 0x1p-48, R = P.pad;
            const double L = fmax(fabs((double)ph[0]), fmax(fabs((double)ph[1]), fabs((double)ph[2])));
            const double eps = P.D * u2 * (90.0 * R * L + 120.0 * R * R) + 2e-11 + u2 * (3.0 * m + 2.0) + 0x1p-52;
            err[i] = (float)(1.01 * eps * S);
        }
    }
    if (terms) {
        unsigned long long cnt = (unsigned long long)m;
        for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(full, cnt, o);
        if (lane == 0 && cnt) atomicAdd(terms, cnt);
    }
}

int gs_field_init(void)
{
    float2 t[65];
    for (int j = -32; j <= 32; j++) {
        const long double v = exp2l((long double)j / 64.0L);
        const float h = (float)v;
        t[j + 32] = make_float2(h, (float)(v - (long double)h));
    }
    GS_CHECK(cudaMemcpyToSymbol(c_dw_exp2, t, sizeof(t)));
    return GS_OK;
}

int gs_field_dw(const GsProblem &P, const uint64_t *d_vkeys, const double *d_points, int64_t n, double *d_phi,
                float *d_err, unsigned long long *d_terms, cudaStream_t st)
{
    if (n <= 0) return GS_OK;
    const double K = P.D * 1.4426950408889634074, LN2 = 0.6931471805599453094;
    DwConst C;
    C.Kh = (float)K;
    C.Kl = (float)(K - (double)C.Kh);
    C.L2h = (float)LN2;
    C.L2l = (float)(LN2 - (double)C.L2h);
    GS_LAUNCH(k_field_dw<4>, (unsigned)((n + 127) / 128), 128, 0, st)(P, d_vkeys, d_points, n, C, d_phi, d_err,
                                                                     d_terms);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// ---------------------------------------------------------------- mixed field
// FP32 values everywhere; where a vertex's bound leaves a decision open (its
// sign relative to c, the inside test of the triangulation; a surface point's
// position) the double-word re-evaluation above, and FP64 where its bound
// still does.
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
__global__ void k_field_scatter(const double *sub_phi, const int64_t *sub_idx, int64_t m, double *phi, float *err)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    phi[sub_idx[t]] = sub_phi[t];
    if (err) err[sub_idx[t]] = 0.f;
}

// mark[v] = 1 where |phi - c| is within 4 bounds (n + 1 entries, last 0)
int gs_field_flag_near(const GsProblem &P, const double *d_phi, const float *d_err, int64_t n, int64_t *d_mark,
                       cudaStream_t st)
{
    if (n <= 0) return GS_OK;
    cudaMemsetAsync(d_mark + n, 0, sizeof(int64_t), st);
    GS_LAUNCH(k_field_flag, (unsigned)((n + 255) / 256), 256, 0, st)(d_phi, d_err, n, P.c, d_mark);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

int gs_field_recompute(const GsProblem &P, const uint64_t *d_vkeys, int64_t n, int64_t *d_mark, double *d_phi,
                       float *d_err, int64_t *n_recomputed, cudaStream_t st)
{
    *n_recomputed = 0;
    if (n <= 0) return GS_OK;
    int64_t *tot = nullptr;
    int rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
    if (!rc) rc = gs_scan_i64(d_mark, n + 1, tot, st);
    int64_t m = 0;
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(&m, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = gs_sync(st);
        if (e != cudaSuccess) rc = gs_fail_cuda(e, "recompute count", __FILE__, __LINE__);
    }
    gs_free(tot, st);
    if (!rc && m > 0) {
        uint64_t *sk = nullptr;
        int64_t *si = nullptr;
        double *sp = nullptr;
        rc = gs_alloc((void **)&sk, sizeof(uint64_t) * (size_t)m, st);
        if (!rc) rc = gs_alloc((void **)&si, sizeof(int64_t) * (size_t)m, st);
        if (!rc) rc = gs_alloc((void **)&sp, sizeof(double) * (size_t)m, st);
        if (!rc) {
            GS_LAUNCH(k_field_gather, (unsigned)((n + 255) / 256), 256, 0, st)(d_mark, n, d_vkeys, sk, si);
            rc = gs_field_f64(P, sk, nullptr, m, sp, nullptr, nullptr, st);
        }
        if (!rc) GS_LAUNCH(k_field_scatter, (unsigned)((m + 255) / 256), 256, 0, st)(sp, si, m, d_phi, d_err);
        gs_free(sk, st); gs_free(si, st); gs_free(sp, st);
    }
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    *n_recomputed = m;
    return GS_OK;
}

__global__ void k_field_scatter_err(const double *sub_phi, const float *sub_err, const int64_t *sub_idx, int64_t m,
                                    double *phi, float *err)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m) return;
    phi[sub_idx[t]] = sub_phi[t];
    err[sub_idx[t]] = sub_err[t];
}

static int read_count(const int64_t *d_tot, int64_t *h, cudaStream_t st, const char *what)
{
    cudaError_t e = cudaMemcpyAsync(h, d_tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = gs_sync(st);
    if (e != cudaSuccess) return gs_fail_cuda(e, what, __FILE__, __LINE__);
    return GS_OK;
}

int gs_field_refine(const GsProblem &P, const uint64_t *d_vkeys, int64_t n, int64_t *d_mark, double *d_phi,
                    float *d_err, int64_t *n_dw, int64_t *n_fp64, cudaStream_t st)
{
    *n_dw = 0;
    *n_fp64 = 0;
    if (n <= 0) return GS_OK;
    int64_t *tot = nullptr;
    int rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
    if (!rc) rc = gs_scan_i64(d_mark, n + 1, tot, st);
    int64_t m = 0, m2 = 0;
    if (!rc) rc = read_count(tot, &m, st, "refine count");
    if (!rc && m > 0) {
        uint64_t *sk = nullptr, *sk2 = nullptr;
        int64_t *si = nullptr, *c2 = nullptr, *si2 = nullptr;
        double *sp = nullptr, *sp2 = nullptr;
        float *se = nullptr;
        rc = gs_alloc((void **)&sk, sizeof(uint64_t) * (size_t)m, st);
        if (!rc) rc = gs_alloc((void **)&si, sizeof(int64_t) * (size_t)m, st);
        if (!rc) rc = gs_alloc((void **)&sp, sizeof(double) * (size_t)m, st);
        if (!rc) rc = gs_alloc((void **)&se, sizeof(float) * (size_t)m, st);
        if (!rc) rc = gs_alloc((void **)&c2, sizeof(int64_t) * (size_t)(m + 1), st);
        if (!rc) GS_LAUNCH(k_field_gather, (unsigned)((n + 255) / 256), 256, 0, st)(d_mark, n, d_vkeys, sk, si);
        if (!rc) rc = gs_field_dw(P, sk, nullptr, m, sp, se, nullptr, st);
        // the sign relative to c still open: FP64
        if (!rc) {
            cudaMemsetAsync(c2 + m, 0, sizeof(int64_t), st);
            GS_LAUNCH(k_field_flag, (unsigned)((m + 255) / 256), 256, 0, st)(sp, se, m, P.c, c2);
            rc = gs_scan_i64(c2, m + 1, tot, st);
        }
        if (!rc) rc = read_count(tot, &m2, st, "refine FP64 count");
        if (!rc && m2 > 0) {
            rc = gs_alloc((void **)&sk2, sizeof(uint64_t) * (size_t)m2, st);
            if (!rc) rc = gs_alloc((void **)&si2, sizeof(int64_t) * (size_t)m2, st);
            if (!rc) rc = gs_alloc((void **)&sp2, sizeof(double) * (size_t)m2, st);
            if (!rc) {
                GS_LAUNCH(k_field_gather, (unsigned)((m + 255) / 256), 256, 0, st)(c2, m, sk, sk2, si2);
                rc = gs_field_f64(P, sk2, nullptr, m2, sp2, nullptr, nullptr, st);
            }
            if (!rc) GS_LAUNCH(k_field_scatter, (unsigned)((m2 + 255) / 256), 256, 0, st)(sp2, si2, m2, sp, se);
        }
        if (!rc) GS_LAUNCH(k_field_scatter_err, (unsigned)((m + 255) / 256), 256, 0, st)(sp, se, si, m, d_phi, d_err);
        gs_free(sk, st); gs_free(si, st); gs_free(sp, st); gs_free(se, st); gs_free(c2, st);
        gs_free(sk2, st); gs_free(si2, st); gs_free(sp2, st);
    }
    gs_free(tot, st);
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    *n_dw = m;
    *n_fp64 = m2;
    return GS_OK;
}

// ---------------------------------------------------------------- adjoint
// dL/dtheta = sum_v lambda_v dphi(v)/dtheta with the field's terms
// recomputed (not stored): for t = exp(-D (|v - x_i|^2 - r_i^2)),
//   dt/dx_i = 2 D t (v - x_i),  dt/dr_i = 2 D t r_i,  dt/dD = -t (|v - x_i|^2 - r_i^2).
// The cutoff sphere moves with r_i and D; its terms are ~cutoff_rel c and
// their jump is not differentiated.
__global__ void __launch_bounds__(128) k_field_adjoint(GsProblem P, const int32_t *__restrict__ perm,
                                                       const uint64_t *vkeys, const double *__restrict__ lambda,
                                                       int64_t n, double *gx, double *gr, double *gD)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double dD = 0.0;
    const double lam = i < n ? lambda[i] : 0.0;
    if (lam != 0.0) {
        double p[3];
        point_of(P, vkeys, nullptr, i, p);
        const double D = P.D, nD = -P.D;
        float ph[3], pl[3];
        for (int a = 0; a < 3; a++) {
            double rel = p[a] - P.origin[a];
            ph[a] = (float)rel;
            pl[a] = (float)(rel - (double)ph[a]);
        }
        gs_for_rows(P, ph, ph, [&](int b, int e, int64_t, int) {
            for (int k = b; k < e; k++) {
                float fx = (ph[0] - P.hx[k]) + (pl[0] - P.lx[k]);
                float fy = (ph[1] - P.hy[k]) + (pl[1] - P.ly[k]);
                float fz = (ph[2] - P.hz[k]) + (pl[2] - P.lz[k]);
                float f2 = fx * fx + fy * fy + fz * fz;
                if (f2 > P.fR2[k] * (1.f + 1e-5f) + 1e-5f) continue;
                double dx = __dsub_rn(p[0], P.ax[k]), dy = __dsub_rn(p[1], P.ay[k]), dz = __dsub_rn(p[2], P.az[k]);
                double d2 = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                if (d2 > P.aR2[k]) continue;
                const double t = P.aw[k] * gs_exp(nD * d2), r = P.ar[k];
                const double s = lam * 2.0 * D * t;
                const int64_t o = perm[k];
                atomicAdd(&gx[3 * o], s * dx);
                atomicAdd(&gx[3 * o + 1], s * dy);
                atomicAdd(&gx[3 * o + 2], s * dz);
                atomicAdd(&gr[o], s * r);
                dD -= lam * t * (d2 - r * r);
            }
        });
    }
    for (int o = 16; o > 0; o >>= 1) dD += __shfl_xor_sync(0xffffffffu, dD, o);
    if ((threadIdx.x & 31) == 0 && dD != 0.0) atomicAdd(gD, dD);
}

int gs_field_adjoint(const GsProblem &P, const int32_t *d_perm, const uint64_t *d_vkeys, const double *d_lambda,
                     int64_t nv, double *d_gx, double *d_gr, double *d_gD, cudaStream_t st)
{
    if (nv <= 0) return GS_OK;
    GS_LAUNCH(k_field_adjoint, (unsigned)((nv + 127) / 128), 128, 0, st)(P, d_perm, d_vkeys, d_lambda, nv, d_gx, d_gr,
                                                                        d_gD);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// lattice values within 1e-10 c of c (the vertex-sign margin): cnt += count
__global__ void k_count_near(const double *__restrict__ v, int64_t n, double c, unsigned long long *cnt)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool nr = i < n && fabs(v[i] - c) < GS_NEAR_REL * c;
    const unsigned b = __ballot_sync(0xffffffffu, nr);
    if ((threadIdx.x & 31) == 0 && b) atomicAdd(cnt, (unsigned long long)__popc(b));
}

int gs_count_near(const double *d_v, int64_t n, double c, unsigned long long *d_cnt, cudaStream_t st)
{
    if (n <= 0) return GS_OK;
    GS_LAUNCH(k_count_near, (unsigned)((n + 255) / 256), 256, 0, st)(d_v, n, c, d_cnt);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}
