// gs_level.cu -- one level of the adaptive partition (section 2.2):
//   * the coefficient tensor A of every examined cube (eqs polynew,
//     tensor1, tensor2): per atom the Legendre projection of its 1-D
//     Gaussian factor on each axis (eqs poly2_1..3, n = 3) with the C0
//     endpoint correction (eqs poly3, condition1, alpha), weighted by
//     exp(D r^2) and accumulated as a rank-one update;
//   * the estimate of [L, U] by the two-level truncated SVD (eqs matrix1,
//     SVD1-SVD7, Sxyz, bound1-bound3) and the decision
//     discard / accept / split (steps 1-3 of section 2.2).
//
// Layout: cubes are examined in octets (the 8 children of one split parent,
// or a 2x2x2 block of root cubes).  One warp accumulates one octet: lane
// (child c = lane/4, j = lane%4) owns the 16 entries A_c[j][*][*].  The 8
// children share the candidate atoms (cell rows around the parent box) and,
// per atom and axis, two child intervals, so each atom's coefficients are
// computed once per octet and used by up to 8 cubes.  Estimation runs one
// thread per cube.
#include <cmath>
#include <cstdio>
#include <vector>

#include "gs_host.cuh"

// ---------------------------------------------------------------- quadrature
// Gauss-Legendre nodes t_k and folded weights W_kj = (2j+1)/2 * w_k * L_j(t_k),
// so that alpha_j = sum_k W_kj f(t_k).  Variants with 8, 12, 16, 24, 6 and 5 nodes.
#define GQ_VARIANTS 6
#define GQ_MAX 24
__constant__ double c_gq_t[GQ_VARIANTS][GQ_MAX];
__constant__ double c_gq_W[GQ_VARIANTS][GQ_MAX][4];
__constant__ float c_gq_tf[GQ_VARIANTS][GQ_MAX];
__constant__ float c_gq_Wf[GQ_VARIANTS][GQ_MAX][4];
static const int kGqN[GQ_VARIANTS] = {8, 12, 16, 24, 6, 5};

// nodes of P_n as eigen-free Newton iteration in long double, started from
// Tricomi's asymptotic estimate
static void gl_rule(int n, long double *t, long double *w)
{
    const long double pi = 3.141592653589793238462643383279502884L;
    for (int k = 1; k <= n; k++) {
        long double th = pi * (4.0L * k - 1.0L) / (4.0L * n + 2.0L);
        long double x = (1.0L - (n - 1.0L) / (8.0L * n * n * n)) * cosl(th);
        long double dp = 0;
        for (int it = 0; it < 60; it++) {
            long double pm1 = 1.0L, p = x;
            for (int m = 2; m <= n; m++) {
                long double pn = ((2.0L * m - 1.0L) * x * p - (m - 1.0L) * pm1) / m;
                pm1 = p;
                p = pn;
            }
            dp = n * (pm1 - x * p) / (1.0L - x * x);
            long double dx = p / dp;
            x -= dx;
            if (fabsl(dx) < 1e-19L) break;
        }
        t[k - 1] = x;
        w[k - 1] = 2.0L / ((1.0L - x * x) * dp * dp);
    }
}

// Re-expansion of a cubic Legendre series on a half interval: for the lower
// (h = 0) or upper (h = 1) half of [-1,1], R[h][p][j] = (2p+1)/2 times the
// integral of L_j((t + sigma)/2) L_p(t) over [-1,1] (sigma = -1 or +1), so
// that the child's coefficients are R times the parent's.
__constant__ double c_reexp[2][4][4];

static bool g_gq_ready[64];

int gs_quadrature_init(void)
{
    int dev = 0;
    GS_CHECK(cudaGetDevice(&dev));
    if (dev >= 0 && dev < 64 && g_gq_ready[dev]) return GS_OK;
    static double t[GQ_VARIANTS][GQ_MAX], W[GQ_VARIANTS][GQ_MAX][4];
    static float tf[GQ_VARIANTS][GQ_MAX], Wf[GQ_VARIANTS][GQ_MAX][4];
    for (int v = 0; v < GQ_VARIANTS; v++) {
        long double tt[GQ_MAX], ww[GQ_MAX];
        int n = kGqN[v];
        gl_rule(n, tt, ww);
        for (int k = 0; k < GQ_MAX; k++) {
            long double x = k < n ? tt[k] : 0.0L, wk = k < n ? ww[k] : 0.0L;
            long double L[4] = {1.0L, x, (3.0L * x * x - 1.0L) / 2.0L, (5.0L * x * x * x - 3.0L * x) / 2.0L};
            t[v][k] = (double)x;
            tf[v][k] = (float)x;
            for (int j = 0; j < 4; j++) {
                W[v][k][j] = (double)((2.0L * j + 1.0L) / 2.0L * wk * L[j]);
                Wf[v][k][j] = (float)W[v][k][j];
            }
        }
    }
    {
        // 4-point Gauss-Legendre integrates the degree-6 products exactly
        long double t4[4], w4[4];
        gl_rule(4, t4, w4);
        auto L = [](int j, long double x) -> long double {
            switch (j) {
            case 0: return 1.0L;
            case 1: return x;
            case 2: return (3.0L * x * x - 1.0L) / 2.0L;
            default: return (5.0L * x * x * x - 3.0L * x) / 2.0L;
            }
        };
        static double R[2][4][4];
        for (int h = 0; h < 2; h++)
            for (int p = 0; p < 4; p++)
                for (int j = 0; j < 4; j++) {
                    long double acc = 0.0L, sg = h ? 1.0L : -1.0L;
                    for (int q = 0; q < 4; q++) acc += w4[q] * L(j, (t4[q] + sg) / 2.0L) * L(p, t4[q]);
                    R[h][p][j] = (double)((2.0L * p + 1.0L) / 2.0L * acc);
                }
        GS_CHECK(cudaMemcpyToSymbol(c_reexp, R, sizeof(R)));
    }
    GS_CHECK(cudaMemcpyToSymbol(c_gq_t, t, sizeof(t)));
    GS_CHECK(cudaMemcpyToSymbol(c_gq_W, W, sizeof(W)));
    GS_CHECK(cudaMemcpyToSymbol(c_gq_tf, tf, sizeof(tf)));
    GS_CHECK(cudaMemcpyToSymbol(c_gq_Wf, Wf, sizeof(Wf)));
    if (dev >= 0 && dev < 64) g_gq_ready[dev] = true;
    return GS_OK;
}

// node count for an interval of half-width hh: the quadrature error of the
// projection stays below ~1e-14 (FP64) for sqrt(D)*hh up to each limit
static int gq_variant(double D, double hh, bool fp32)
{
    double a = sqrt(D) * hh;
    // FP32: quadrature error of each coefficient below 2e-7 of the Gaussian's
    // peak (5 nodes: 3e-8 up to a = 0.2; 6 nodes: 2e-7 up to 0.5)
    if (fp32) return a <= 0.2 ? 5 : (a <= 0.5 ? 4 : (a <= 1.0 ? 0 : (a <= 1.5 ? 1 : 2)));
    if (a <= 0.25) return 0;
    if (a <= 0.75) return 1;
    if (a <= 1.0) return 2;
    return 3;
}

// ---------------------------------------------------------------- octet geometry
struct Octet {
    int64_t I, J, K;   // parent coords (children at 2I+dx, ...)
    uint8_t vmask;     // valid children
};

__device__ __forceinline__ Octet octet_of(const GsProblem &P, int level, const uint64_t *parents,
                                          const uint8_t *vmask, int64_t o)
{
    Octet q;
    if (parents) {
        uint64_t k = parents[o];
        q.I = gk_x(k); q.J = gk_y(k); q.K = gk_z(k);
        q.vmask = vmask ? vmask[o] : 0xFF;
        if (level == 0) {
            // root blocks: drop children outside the root grid
            for (int c = 0; c < 8; c++) {
                int64_t x = 2 * q.I + (c & 1), y = 2 * q.J + ((c >> 1) & 1), z = 2 * q.K + (c >> 2);
                if (x >= P.nroot[0] || y >= P.nroot[1] || z >= P.nroot[2]) q.vmask &= (uint8_t)~(1u << c);
            }
        }
    } else {
        // root blocks of 2x2x2 cubes, x fastest
        int64_t bx = (P.nroot[0] + 1) / 2, by = (P.nroot[1] + 1) / 2;
        q.I = o % bx;
        q.J = (o / bx) % by;
        q.K = o / (bx * by);
        uint8_t m = 0;
        for (int c = 0; c < 8; c++) {
            int64_t x = 2 * q.I + (c & 1), y = 2 * q.J + ((c >> 1) & 1), z = 2 * q.K + (c >> 2);
            if (x < P.nroot[0] && y < P.nroot[1] && z < P.nroot[2]) m |= (uint8_t)(1u << c);
        }
        q.vmask = m;
    }
    return q;
}

// ---------------------------------------------------------------- FP64 accumulate
#define ACC_WARPS 4
#define ACC_Q 64

// one axis: C0-corrected Legendre coefficients of exp(-D (x - xi)^2) on
// [e0,e1] and [e1,e2] (the two child intervals), FP64; `need` selects the
// intervals (bit 0: [e0,e1], bit 1: [e1,e2]) some accumulated child uses
template <int GV, int NQ>
__device__ __forceinline__ void axis_coeffs_f64(double xi, double e0, double e1, double e2, double D,
                                                double *out /* [2][4] */, int need = 3)
{
    const int gv = GV, nq = NQ;
    double f0 = (need & 1) ? gs_exp(-D * (e0 - xi) * (e0 - xi)) : 0.0;
    double f1 = gs_exp(-D * (e1 - xi) * (e1 - xi));
    double f2 = (need & 2) ? gs_exp(-D * (e2 - xi) * (e2 - xi)) : 0.0;
#pragma unroll
    for (int h = 0; h < 2; h++) {
        if (!((need >> h) & 1)) continue;
        double lo = h ? e1 : e0, hi = h ? e2 : e1;
        double m = __dmul_rn(0.5, __dadd_rn(lo, hi)) - xi, hh = __dmul_rn(0.5, __dsub_rn(hi, lo));
        double a0 = 0, a1 = 0, a2 = 0, a3 = 0;
#pragma unroll
        for (int k = 0; k < nq; k++) {
            double d = fma(hh, c_gq_t[gv][k], m);
            double f = gs_exp(-D * d * d);
            a0 = fma(c_gq_W[gv][k][0], f, a0);
            a1 = fma(c_gq_W[gv][k][1], f, a1);
            a2 = fma(c_gq_W[gv][k][2], f, a2);
            a3 = fma(c_gq_W[gv][k][3], f, a3);
        }
        double fa = h ? f1 : f0, fb = h ? f2 : f1;
        double eR = fb - (a0 + a1 + a2 + a3);
        double eL = fa - (a0 - a1 + a2 - a3);
        out[4 * h + 0] = a0;
        out[4 * h + 1] = a1;
        out[4 * h + 2] = a2 + 0.5 * (eR + eL);
        out[4 * h + 3] = a3 + 0.5 * (eR - eL);
    }
}

// BATCH: octet o belongs to molecule mol[o], whose problem is probs[mol[o]]
// (the molecules of one launch share D, so one quadrature rule serves all)
template <int GV, int NQ, bool BATCH>
__global__ void __launch_bounds__(32 * ACC_WARPS) k_accum_f64(GsProblem P0, int level, const uint64_t *parents,
                                                               const uint8_t *vmask, int64_t n_oct,
                                                               double pad, double *__restrict__ A_out,
                                                               unsigned long long *pairs, unsigned *status,
                                                               const GsProblem *__restrict__ probs,
                                                               const int32_t *__restrict__ mol)
{
    __shared__ double s_cf[ACC_WARPS][32][25];   // per queued atom: 3 axes x 2 intervals x 4, then w
    __shared__ int s_qi[ACC_WARPS][ACC_Q];
    __shared__ uint8_t s_qm[ACC_WARPS][ACC_Q];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    unsigned long long my_pairs = 0;
    for (int64_t o = (int64_t)blockIdx.x * ACC_WARPS + wl; o < n_oct; o += (int64_t)gridDim.x * ACC_WARPS) {
        const GsProblem &P = BATCH ? probs[mol[o]] : P0;
        Octet q = octet_of(P, level, parents, vmask, o);
        int64_t base[3] = {2 * q.I, 2 * q.J, 2 * q.K};
        double e[3][3];
        float eh[3][3], el[3][3];
        for (int a = 0; a < 3; a++)
            for (int t = 0; t < 3; t++) {
                e[a][t] = gs_lat(P, a, base[a] + t, level);
                double rel = e[a][t] - P.origin[a];
                eh[a][t] = (float)rel;
                el[a][t] = (float)(rel - (double)eh[a][t]);
            }
        double acc[16];
#pragma unroll
        for (int t = 0; t < 16; t++) acc[t] = 0.0;
        int qn = 0;
        const uint8_t vm = q.vmask;
        // update lanes: 4 per (accumulated child, x index); when at most four
        // children are accumulated (a recheck of some cubes of the octet),
        // G groups of lanes take every G-th queued atom and their sums are
        // added at the end, so the FP64 updates issue for several atoms at once
        const int nc = __popc(vm);
        const int gsz = nc <= 1 ? 4 : (nc <= 2 ? 8 : (nc <= 4 ? 16 : 32)), G = 32 / gsz;
        const int pg = lane / gsz, slot = (lane % gsz) >> 2, j = lane & 3;
        int c = -1;
        for (int cc = 0, k = 0; cc < 8; cc++)
            if ((vm >> cc) & 1) {
                if (k == slot) c = gsz == 32 ? (lane >> 2) : cc;
                k++;
            }
        if (gsz == 32) c = lane >> 2;   // every child has its lanes (as without grouping)
        const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;

        // intervals used by the selected children, per axis
        int need[3] = {0, 0, 0};
        for (int cc = 0; cc < 8; cc++)
            if ((vm >> cc) & 1) {
                need[0] |= 1 << (cc & 1);
                need[1] |= 1 << ((cc >> 1) & 1);
                need[2] |= 1 << (cc >> 2);
            }
        auto process = [&](int nproc) {
            if (lane < nproc) {
                int i = s_qi[wl][lane];
                double xs[3] = {P.ax[i], P.ay[i], P.az[i]};
                for (int a = 0; a < 3; a++)
                    axis_coeffs_f64<GV, NQ>(xs[a], e[a][0], e[a][1], e[a][2], P.D, &s_cf[wl][lane][8 * a], need[a]);
                s_cf[wl][lane][24] = P.aw[i];
            }
            __syncwarp();
            for (int t = pg; t < nproc; t += G) {
                if (c >= 0 && ((s_qm[wl][t] >> c) & 1)) {
                    const double *cf = s_cf[wl][t];
                    double wa = cf[24] * cf[4 * cx + j];
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        double wb = wa * cf[8 + 4 * cy + k];
#pragma unroll
                        for (int l = 0; l < 4; l++) acc[4 * k + l] = fma(wb, cf[16 + 4 * cz + l], acc[4 * k + l]);
                    }
                }
            }
            __syncwarp();
        };

        // membership of one candidate per lane (i < 0: none): FP32 box
        // distance with a margin, the exact FP64 test (the definition) inside
        // the margin
        auto filter = [&](int i) {
            unsigned m = 0;
            if (i >= 0) {
                const float ah[3] = {P.hx[i], P.hy[i], P.hz[i]}, al[3] = {P.lx[i], P.ly[i], P.lz[i]};
                float g2[3][2];
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int hI = 0; hI < 2; hI++) {
                        float dlo = (eh[a][hI] - ah[a]) + (el[a][hI] - al[a]);
                        float dhi = (ah[a] - eh[a][hI + 1]) + (al[a] - el[a][hI + 1]);
                        float g = fmaxf(0.f, fmaxf(dlo, dhi));
                        g2[a][hI] = g * g;
                    }
                const float R2 = P.fR2[i];
                const float tol = 1e-5f * R2 + 1e-5f;
                unsigned nearm = 0;
#pragma unroll
                for (int cc = 0; cc < 8; cc++) {
                    float d2 = g2[0][cc & 1] + g2[1][(cc >> 1) & 1] + g2[2][cc >> 2];
                    if (d2 < R2 - tol) m |= 1u << cc;
                    else if (d2 <= R2 + tol) nearm |= 1u << cc;
                }
                m &= vm;
                nearm &= vm;
                while (nearm) {
                    const int cc = __ffs(nearm) - 1;
                    nearm &= nearm - 1;
                    double x = P.ax[i], y = P.ay[i], z = P.az[i];
                    double dx = gs_axis_gap(e[0][cc & 1], e[0][(cc & 1) + 1], x);
                    double dy = gs_axis_gap(e[1][(cc >> 1) & 1], e[1][((cc >> 1) & 1) + 1], y);
                    double dz = gs_axis_gap(e[2][cc >> 2], e[2][(cc >> 2) + 1], z);
                    double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                    if (dd <= P.aR2[i]) m |= 1u << cc;
                }
            }
            my_pairs += __popc(m);
            unsigned bal = __ballot_sync(0xffffffffu, m != 0);
            int pos = qn + __popc(bal & below);
            if (m) { s_qi[wl][pos] = i; s_qm[wl][pos] = (uint8_t)m; }
            qn += __popc(bal);
            __syncwarp();
            if (qn >= 32) {
                process(32);
                int rest = qn - 32;
                int mi = 0; uint8_t mm = 0;
                if (lane < rest) { mi = s_qi[wl][32 + lane]; mm = s_qm[wl][32 + lane]; }
                __syncwarp();
                if (lane < rest) { s_qi[wl][lane] = mi; s_qm[wl][lane] = mm; }
                __syncwarp();
                qn = rest;
            }
        };

        if (vm) {
            float flo[3] = {eh[0][0], eh[1][0], eh[2][0]}, fhi[3] = {eh[0][2], eh[1][2], eh[2][2]};
            gs_warp_candidates(P, flo, fhi, lane, filter);
            if (qn > 0) process(qn);
        }
        for (int off = gsz; off < 32; off <<= 1)
#pragma unroll
            for (int t = 0; t < 16; t++) acc[t] += __shfl_xor_sync(0xffffffffu, acc[t], off);
        if (pg == 0 && c >= 0) {
            double *dst = A_out + ((size_t)o * 8 + c) * 64 + 16 * j;
#pragma unroll
            for (int t = 0; t < 16; t++) dst[t] = acc[t];
        }
        if (gsz < 32)   // the children not accumulated hold zeros, as with one lane group
            for (int cc = 0; cc < 8; cc++)
                if (!((vm >> cc) & 1)) {
                    double *z = A_out + ((size_t)o * 8 + cc) * 64;
                    z[lane] = 0.0;
                    z[32 + lane] = 0.0;
                }
    }
    if (pairs) {
        for (int off = 16; off > 0; off >>= 1) my_pairs += __shfl_xor_sync(0xffffffffu, my_pairs, off);
        if (lane == 0 && my_pairs) atomicAdd(pairs, my_pairs);
    }
    (void)status;
    (void)pad;
}

static int grid_for(int64_t n_items, int per_block)
{
    int64_t b = (n_items + per_block - 1) / per_block;
    int64_t cap = 152LL * 64;
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

int gs_accum_f64(const GsProblem &P, int level, const uint64_t *d_parents, const uint8_t *d_vmask, int64_t n_oct,
                 double *d_A, unsigned long long *d_pairs, unsigned *d_status, cudaStream_t st, float *ms,
                 const GsProblem *d_probs, const int32_t *d_mol)
{
    if (n_oct <= 0) return GS_OK;
    double h = gs_h(P, level);
    int gv = gq_variant(P.D, 0.5 * h, false);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) { cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventRecord(e0, st); }
    const unsigned grid = grid_for(n_oct, ACC_WARPS);
#define GS_ACC64(V, N)                                                                                              \
    do {                                                                                                            \
        if (d_probs)                                                                                                \
            GS_LAUNCH((k_accum_f64<V, N, true>), grid, 32 * ACC_WARPS, 0, st)(P, level, d_parents, d_vmask, n_oct,  \
                                                                             P.pad, d_A, d_pairs, d_status,         \
                                                                             d_probs, d_mol);                       \
        else                                                                                                        \
            GS_LAUNCH((k_accum_f64<V, N, false>), grid, 32 * ACC_WARPS, 0, st)(P, level, d_parents, d_vmask, n_oct, \
                                                                              P.pad, d_A, d_pairs, d_status,        \
                                                                              nullptr, nullptr);                    \
    } while (0)
    switch (gv) {
    case 0: GS_ACC64(0, 8); break;
    case 1: GS_ACC64(1, 12); break;
    case 2: GS_ACC64(2, 16); break;
    default: GS_ACC64(3, 24); break;
    }
#undef GS_ACC64
    if (ms) {
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        *ms += t;
        cudaEventDestroy(e0); cudaEventDestroy(e1);
    }
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// ---------------------------------------------------------------- estimation
// Truncated SVD bounds of section 2.2.2, templated on the arithmetic type.

template <typename T> __device__ __forceinline__ T t_sqrt(T x);
template <> __device__ __forceinline__ double t_sqrt<double>(double x) { return sqrt(x); }
template <> __device__ __forceinline__ float t_sqrt<float>(float x) { return sqrtf(x); }
template <typename T> __device__ __forceinline__ T t_abs(T x) { return x < T(0) ? -x : x; }
template <typename T> struct Eps;
// Jacobi rotation zeroing the inner product ga of two rows with squared
// norms al, be; false when the rows are already orthogonal to within Eps
template <typename T> __device__ __forceinline__ bool jac_rot(T al, T be, T ga, T &cs, T &sn);
template <> struct Eps<double> { static __device__ __forceinline__ double v() { return 1e-15; } };
// FP32: the rounding noise of a 16-term dot product is ~1e-6 of |p||q|, so a
// tighter rotation threshold would keep rotating noise until the sweep limit
template <> struct Eps<float> { static __device__ __forceinline__ float v() { return 1e-6f; } };

template <> __device__ __forceinline__ bool jac_rot<double>(double al, double be, double ga, double &cs, double &sn)
{
    if (ga == 0.0 || fabs(ga) <= Eps<double>::v() * sqrt(al * be)) return false;
    double tau = (be - al) / (2.0 * ga);
    double t = (tau >= 0.0 ? 1.0 : -1.0) / (fabs(tau) + sqrt(1.0 + tau * tau));
    cs = 1.0 / sqrt(1.0 + t * t);
    sn = cs * t;
    return true;
}
// FP32: the rotation only has to reduce ga (the sweep repeats until the
// threshold holds), so the approximate reciprocal, divide and square roots
// of the SFU suffice
template <> __device__ __forceinline__ bool jac_rot<float>(float al, float be, float ga, float &cs, float &sn)
{
    const float e = Eps<float>::v();
    if (ga == 0.f || ga * ga <= e * e * (al * be)) return false;
    float tau = __fdividef(be - al, 2.f * ga);
    const float at = fabsf(tau);
    float t;
    if (at > 1e18f) {
        t = 0.5f / at;   // 1 / (|tau| + sqrt(1 + tau^2)) without overflowing tau^2
    } else {
        const float q = 1.f + at * at;
        t = __fdividef(1.f, at + q * rsqrtf(q));
    }
    t = copysignf(t, tau);
    cs = rsqrtf(1.f + t * t);
    sn = cs * t;
    return true;
}

// one-sided Jacobi on the 4 rows of X (4 x N): afterwards the rows are
// orthogonal and X_in = Q^T X_out.  Returns singular values sorted
// descending in s, with the matching left vectors (rows of Q) in u and the
// right vectors (normalised rows of X) written back into X in sorted order.
template <typename T, int N>
__device__ void jacobi4(T (&X)[4][N], T (&s)[4], T (&u)[4][4])
{
    T Q[4][4];
#pragma unroll
    for (int a = 0; a < 4; a++)
#pragma unroll
        for (int b = 0; b < 4; b++) Q[a][b] = a == b ? T(1) : T(0);
    for (int sweep = 0; sweep < 40; sweep++) {
        bool any = false;
#pragma unroll
        for (int p = 0; p < 3; p++)
#pragma unroll
            for (int q = p + 1; q < 4; q++) {
                T al = 0, be = 0, ga = 0;
                if constexpr (sizeof(T) == 4 && N % 4 == 0) {
                    // FP32: paired (f32x2) products over k = (2m, 2m+1), two
                    // partial sums each to shorten the dependency chains
                    float2 a2[2] = {make_float2(0.f, 0.f), make_float2(0.f, 0.f)};
                    float2 b2[2] = {a2[0], a2[0]}, g2[2] = {a2[0], a2[0]};
#pragma unroll
                    for (int m = 0; m < N / 2; m++) {
                        const float2 xp = make_float2(X[p][2 * m], X[p][2 * m + 1]);
                        const float2 xq = make_float2(X[q][2 * m], X[q][2 * m + 1]);
                        a2[m & 1] = __ffma2_rn(xp, xp, a2[m & 1]);
                        b2[m & 1] = __ffma2_rn(xq, xq, b2[m & 1]);
                        g2[m & 1] = __ffma2_rn(xp, xq, g2[m & 1]);
                    }
                    const float2 a = __fadd2_rn(a2[0], a2[1]), b = __fadd2_rn(b2[0], b2[1]), g = __fadd2_rn(g2[0], g2[1]);
                    al = a.x + a.y;
                    be = b.x + b.y;
                    ga = g.x + g.y;
                } else {
#pragma unroll
                    for (int k = 0; k < N; k++) {
                        al += X[p][k] * X[p][k];
                        be += X[q][k] * X[q][k];
                        ga += X[p][k] * X[q][k];
                    }
                }
                T cs, sn;
                if (!jac_rot<T>(al, be, ga, cs, sn)) continue;
                any = true;
                if constexpr (sizeof(T) == 4 && N % 2 == 0) {
                    const float2 c2 = make_float2(cs, cs), s2 = make_float2(sn, sn), ns2 = make_float2(-sn, -sn);
#pragma unroll
                    for (int m = 0; m < N / 2; m++) {
                        const float2 xp = make_float2(X[p][2 * m], X[p][2 * m + 1]);
                        const float2 xq = make_float2(X[q][2 * m], X[q][2 * m + 1]);
                        const float2 np2 = __ffma2_rn(c2, xp, __fmul2_rn(ns2, xq));
                        const float2 nq2 = __ffma2_rn(s2, xp, __fmul2_rn(c2, xq));
                        X[p][2 * m] = np2.x; X[p][2 * m + 1] = np2.y;
                        X[q][2 * m] = nq2.x; X[q][2 * m + 1] = nq2.y;
                    }
#pragma unroll
                    for (int m = 0; m < 2; m++) {
                        const float2 qp = make_float2(Q[p][2 * m], Q[p][2 * m + 1]);
                        const float2 qq = make_float2(Q[q][2 * m], Q[q][2 * m + 1]);
                        const float2 np2 = __ffma2_rn(c2, qp, __fmul2_rn(ns2, qq));
                        const float2 nq2 = __ffma2_rn(s2, qp, __fmul2_rn(c2, qq));
                        Q[p][2 * m] = np2.x; Q[p][2 * m + 1] = np2.y;
                        Q[q][2 * m] = nq2.x; Q[q][2 * m + 1] = nq2.y;
                    }
                } else {
#pragma unroll
                    for (int k = 0; k < N; k++) {
                        T xp = X[p][k], xq = X[q][k];
                        X[p][k] = cs * xp - sn * xq;
                        X[q][k] = sn * xp + cs * xq;
                    }
#pragma unroll
                    for (int k = 0; k < 4; k++) {
                        T qp = Q[p][k], qq = Q[q][k];
                        Q[p][k] = cs * qp - sn * qq;
                        Q[q][k] = sn * qp + cs * qq;
                    }
                }
            }
        if (!any) break;
    }
    T sv[4];
    int ord[4] = {0, 1, 2, 3};
#pragma unroll
    for (int p = 0; p < 4; p++) {
        T n2 = 0;
#pragma unroll
        for (int k = 0; k < N; k++) n2 += X[p][k] * X[p][k];
        sv[p] = t_sqrt(n2);
    }
    T Y[4][N];
    if constexpr (sizeof(T) == 4) {
        // stable sort by descending value: row p goes to position pos[p] (the
        // number of rows before it in that order); moves with static indices
        // only, so that X, Q stay in registers
        int pos[4];
#pragma unroll
        for (int p = 0; p < 4; p++) {
            int r = 0;
#pragma unroll
            for (int q = 0; q < 4; q++) r += (sv[q] > sv[p] || (sv[q] == sv[p] && q < p)) ? 1 : 0;
            pos[p] = r;
        }
        (void)ord;
#pragma unroll
        for (int p = 0; p < 4; p++) {
            T inv = sv[p] > T(0) ? T(1) / sv[p] : T(0);
#pragma unroll
            for (int k = 0; k < N; k++) X[p][k] *= inv;
        }
#pragma unroll
        for (int i = 0; i < 4; i++) {
#pragma unroll
            for (int p = 0; p < 4; p++) {
                if (pos[p] != i) continue;
                s[i] = sv[p];
#pragma unroll
                for (int k = 0; k < 4; k++) u[i][k] = Q[p][k];
#pragma unroll
                for (int k = 0; k < N; k++) Y[i][k] = X[p][k];
            }
        }

    } else {
        // stable insertion sort of 4 indices by descending value
        for (int i = 1; i < 4; i++) {
            int o = ord[i], k = i - 1;
            while (k >= 0 && sv[ord[k]] < sv[o]) { ord[k + 1] = ord[k]; k--; }
            ord[k + 1] = o;
        }
        for (int i = 0; i < 4; i++) {
            int p = ord[i];
            s[i] = sv[p];
            T inv = sv[p] > T(0) ? T(1) / sv[p] : T(0);
#pragma unroll
            for (int k = 0; k < 4; k++) u[i][k] = Q[p][k];
#pragma unroll
            for (int k = 0; k < N; k++) Y[i][k] = X[p][k] * inv;
        }
    }
#pragma unroll
    for (int i = 0; i < 4; i++)
#pragma unroll
        for (int k = 0; k < N; k++) X[i][k] = Y[i][k];
}

// range of sum_j c_j L_j(t) over [-1,1]
template <typename T>
__device__ __forceinline__ void cubic_range(const T *cf, T &lo, T &hi)
{
    T p1 = cf[0] + cf[1] + cf[2] + cf[3], m1 = cf[0] - cf[1] + cf[2] - cf[3];
    lo = p1 < m1 ? p1 : m1;
    hi = p1 < m1 ? m1 : p1;
    // derivative 3 b3 t^2 + 2 b2 t + b1 in monomials of the cubic
    T b0 = cf[0] - T(0.5) * cf[2], b1 = cf[1] - T(1.5) * cf[3], b2 = T(1.5) * cf[2], b3 = T(2.5) * cf[3];
    T qa = T(3) * b3, qb = T(2) * b2, qc = b1;
    T r[2];
    int nr = 0;
    if (qa == T(0)) {
        if (qb != T(0)) r[nr++] = -qc / qb;
    } else {
        T disc = qb * qb - T(4) * qa * qc;
        if (disc >= T(0)) {
            T sq = t_sqrt(disc);
            T w = qb >= T(0) ? -(qb + sq) / T(2) : -(qb - sq) / T(2);
            if (w != T(0)) { r[nr++] = w / qa; r[nr++] = qc / w; }
            else r[nr++] = T(0);
        }
    }
    for (int i = 0; i < nr; i++) {
        T t = r[i];
        if (t > T(-1) && t < T(1)) {
            T v = b0 + t * (b1 + t * (b2 + t * b3));
            lo = v < lo ? v : lo;
            hi = v > hi ? v : hi;
        }
    }
}

template <typename T>
__device__ __forceinline__ int rank99(const T (&s)[4], T &margin)
{
    T tot = s[0] + s[1] + s[2] + s[3];
    T acc = 0;
    T thr = T(0.99) * tot;
    int r = 4;
    margin = tot;
    for (int j = 0; j < 4; j++) {
        acc += s[j];
        T m = t_abs(acc - thr);
        margin = m < margin ? m : margin;
        if (acc >= thr) { r = j + 1; break; }
    }
    return r;
}

// Where the 99% rules could go the other way.  A rule j compares
// sum_{i<=j} s_i with 0.99 sum s; the rules that decide the rank are those up
// to the chosen one, and the one after it (if the chosen rule flipped, the
// next one would decide).  RankNear records the rule nearest its threshold,
// the rank it would give if it flipped, and the second-smallest distance.
template <typename T>
struct RankNear {
    T m1, m2;      // smallest and second-smallest distance of a rule from its threshold
    int who;       // -1: outer rule; i >= 0: inner rule of kept term i
    int alt;       // rank that rule gives if it flips (0: none)
    T ssum;        // sum of the outer singular values
};

template <typename T>
__device__ __forceinline__ void rank_near(const T (&s)[4], int r, int who, RankNear<T> &rn)
{
    T tot = s[0] + s[1] + s[2] + s[3];
    T acc = 0;
    T thr = T(0.99) * tot;
    for (int j = 0; j < 4 && j <= r; j++) {
        acc += s[j];
        T m = t_abs(acc - thr);
        // flipping rule j: below -> rank j+1; at or above -> the next rule decides
        int alt = acc >= thr ? j + 2 : j + 1;
        if (j == 3) alt = 0;
        if (m < rn.m1) {
            rn.m2 = rn.m1;
            rn.m1 = m;
            rn.who = who;
            rn.alt = alt > 4 ? 0 : alt;
        } else if (m < rn.m2) {
            rn.m2 = m;
        }
    }
}

// bounds: out = (L, U, sum|R|, sum|high|, rank, inner ranks); rmargin = the
// smallest distance of a rank rule from its 99% threshold
template <typename T>
__device__ __forceinline__ T gap_sens(const T (&s)[4], int kept)
{
    // sum over the kept values of s_i / (distance to the nearest other
    // value): a perturbation E turns the i-th singular pair by about
    // |E| / gap_i, which moves that term's share of the bounds by about
    // s_i |E| / gap_i.  Terms far smaller than their gap contribute little.
    T r = T(0);
    for (int i = 0; i < kept && i < 4; i++) {
        T g = T(1e30);
        if (i > 0) g = s[i - 1] - s[i];
        if (i < 3) { T d = s[i] - s[i + 1]; g = d < g ? d : g; }
        r += s[i] / (g > T(0) ? g : T(1e-30));
    }
    return r < T(1e6) ? r : T(1e6);
}

// fo > 0 forces the outer rank; fi >= 0 forces the inner rank of kept term
// fi to fj; rn (nullable) collects the rules near their thresholds
template <typename T>
__device__ __forceinline__ void estimate_bounds_sens(const T *A, T *out, T &rmargin, T &sens, int fo = 0, int fi = -1,
                                                     int fj = 0, RankNear<T> *rn = nullptr, T *rrel = nullptr);

template <typename T>
__device__ void estimate_bounds(const T *A, T *out, T &rmargin)
{
    T sens;
    estimate_bounds_sens<T>(A, out, rmargin, sens);
}

// element i of four (static indices only, so that arrays stay in registers)
template <typename T>
__device__ __forceinline__ T sel4(int i, T a0, T a1, T a2, T a3)
{
    return i == 0 ? a0 : (i == 1 ? a1 : (i == 2 ? a2 : a3));
}

// rrel (nullable): the smallest distance of a rank rule from its threshold
// relative to its own singular-value sum (outer and inner rules).  The loops
// over kept terms are rolled, each term's row picked by static selects: one
// copy of the inner SVD and bound code instead of one per possible rank,
// which keeps the kernel within the instruction cache.
template <typename T>
__device__ __forceinline__ void estimate_bounds_sens(const T *A, T *out, T &rmargin, T &sens, int fo, int fi, int fj,
                                                     RankNear<T> *rn, T *rrel)
{
    T X[4][16];
    T high = 0, tot = 0;
#pragma unroll
    for (int j = 0; j < 4; j++)
#pragma unroll
        for (int k = 0; k < 16; k++) {
            T v = A[16 * j + k];
            X[j][k] = v;
            tot += t_abs(v);
            if (j >= 2 || (k >> 2) >= 2 || (k & 3) >= 2) high += t_abs(v);
        }
    out[3] = high;
    rmargin = T(1e30);
    sens = T(0);
    if (tot == T(0)) { out[0] = out[1] = out[2] = 0; out[4] = 0; out[5] = 0; return; }
    T s[4], u[4][4];
    jacobi4<T, 16>(X, s, u);
    T rm;
    int jr = rank99(s, rm);
    if (rrel) *rrel = rm / (s[0] + s[1] + s[2] + s[3]);
    if (fo > 0) {
        jr = fo;
        rm = T(1e30);
    } else if (rn) {
        rn->ssum = s[0] + s[1] + s[2] + s[3];
        rank_near<T>(s, jr, -1, *rn);
    }
    rmargin = rm;
    sens = gap_sens<T>(s, jr);
    // R = A minus the kept rank-one terms, subtracted in place
    T R[64];
#pragma unroll
    for (int t = 0; t < 64; t++) R[t] = A[t];
    T M = 0, m = 0;
    int inner = 0;
#pragma unroll 1
    for (int i = 0; i < jr; i++) {
        T V[4][4], d[4], w[4][4], ui[4];
#pragma unroll
        for (int k = 0; k < 4; k++)
#pragma unroll
            for (int l = 0; l < 4; l++) V[k][l] = sel4(i, X[0][4 * k + l], X[1][4 * k + l], X[2][4 * k + l], X[3][4 * k + l]);
#pragma unroll
        for (int a = 0; a < 4; a++) ui[a] = sel4(i, u[0][a], u[1][a], u[2][a], u[3][a]);
        const T si0 = sel4(i, s[0], s[1], s[2], s[3]);
        jacobi4<T, 4>(V, d, w);
        T rmi;
        int ji = rank99(d, rmi);
        if (rrel) {
            const T rr = rmi / (d[0] + d[1] + d[2] + d[3]);
            *rrel = rr < *rrel ? rr : *rrel;
        }
        if (i == fi) {
            ji = fj;
        } else {
            rmargin = rmi < rmargin ? rmi : rmargin;
            if (rn) rank_near<T>(d, ji, i, *rn);
        }
        T si = gap_sens<T>(d, ji);
        sens = si > sens ? si : sens;
        inner += ji;
        T Myz = 0, myz = 0;
#pragma unroll 1
        for (int k = 0; k < ji; k++) {
            T wk[4], Vk[4];
#pragma unroll
            for (int b = 0; b < 4; b++) {
                wk[b] = sel4(k, w[0][b], w[1][b], w[2][b], w[3][b]);
                Vk[b] = sel4(k, V[0][b], V[1][b], V[2][b], V[3][b]);
            }
            const T dk = sel4(k, d[0], d[1], d[2], d[3]);
            T ly, hy, lz, hz;
            cubic_range(wk, ly, hy);
            cubic_range(Vk, lz, hz);
            T p0 = hy * hz, p1 = hy * lz, p2 = ly * hz, p3 = ly * lz;
            T pmx = p0, pmn = p0;
            pmx = p1 > pmx ? p1 : pmx; pmn = p1 < pmn ? p1 : pmn;
            pmx = p2 > pmx ? p2 : pmx; pmn = p2 < pmn ? p2 : pmn;
            pmx = p3 > pmx ? p3 : pmx; pmn = p3 < pmn ? p3 : pmn;
            Myz += dk * pmx;
            myz += dk * pmn;
            T sd = si0 * dk;
#pragma unroll
            for (int a = 0; a < 4; a++) {
                T sa = sd * ui[a];
#pragma unroll
                for (int b = 0; b < 4; b++) {
                    T sab = sa * wk[b];
#pragma unroll
                    for (int cc = 0; cc < 4; cc++) R[16 * a + 4 * b + cc] -= sab * Vk[cc];
                }
            }
        }
        T lx, hx;
        cubic_range(ui, lx, hx);
        T p0 = hx * Myz, p1 = hx * myz, p2 = lx * Myz, p3 = lx * myz;
        T pmx = p0, pmn = p0;
        pmx = p1 > pmx ? p1 : pmx; pmn = p1 < pmn ? p1 : pmn;
        pmx = p2 > pmx ? p2 : pmx; pmn = p2 < pmn ? p2 : pmn;
        pmx = p3 > pmx ? p3 : pmx; pmn = p3 < pmn ? p3 : pmn;
        M += si0 * pmx;
        m += si0 * pmn;
    }
    T sr = 0;
#pragma unroll
    for (int t = 0; t < 64; t++) sr += t_abs(R[t]);
    out[0] = m - sr;
    out[1] = M + sr;
    out[2] = sr;
    out[4] = (T)jr;
    out[5] = (T)inner;
}

template <typename T>
__device__ __forceinline__ int decide(const T *b, T c, T precision, int level, int max_depth)
{
    if (b[4] == T(0)) return DEC_DISCARD;
    if (!(b[0] <= c && c <= b[1])) return DEC_DISCARD;
    if (b[3] <= precision) return DEC_ACCEPT;
    if (level >= max_depth) return DEC_FORCED;
    return DEC_SPLIT;
}

// P~ at the 8 cube corners: L_n(+-1) = (+-1)^n, so each corner value is a
// signed sum of the coefficients; lo and hi receive the smallest and largest
template <typename T>
__device__ __forceinline__ void corner_range(const T *a, T &lo, T &hi)
{
    lo = T(3.0e38);
    hi = T(-3.0e38);
#pragma unroll
    for (int sx = 0; sx < 2; sx++) {
        T bx[16];
#pragma unroll
        for (int kl = 0; kl < 16; kl++) {
            const T e = a[kl] + a[32 + kl], o = a[16 + kl] + a[48 + kl];
            bx[kl] = sx ? e + o : e - o;
        }
#pragma unroll
        for (int sy = 0; sy < 2; sy++) {
            T cz[4];
#pragma unroll
            for (int l = 0; l < 4; l++) {
                const T e = bx[l] + bx[8 + l], o = bx[4 + l] + bx[12 + l];
                cz[l] = sy ? e + o : e - o;
            }
            const T e = cz[0] + cz[2], o = cz[1] + cz[3];
            lo = fmin(lo, fmin(e - o, e + o));
            hi = fmax(hi, fmax(e - o, e + o));
        }
    }
}

// Literal order of steps 2 and 3: a child whose higher-order coefficients
// meet the bound is accepted before its bounds are tested; a root cube that
// passes the bound test is divided.
__device__ __forceinline__ int decide_literal(const double *b, double c, double precision, int level, int max_depth)
{
    if (b[4] == 0.0) return DEC_DISCARD;
    if (level > 0 && b[3] <= precision) return DEC_ACCEPT;
    if (!(b[0] <= c && c <= b[1])) return DEC_DISCARD;
    if (level >= max_depth) return DEC_FORCED;
    return DEC_SPLIT;
}

// size of the higher-than-linear coefficients: largest magnitude (GS_NORM_MAX)
// or root sum of squares (GS_NORM_RSS); the sum of magnitudes is b[3] already
__device__ __forceinline__ double high_norm(const double *a, int norm)
{
    double mx = 0.0, ss = 0.0;
    for (int j = 0; j < 4; j++)
        for (int k = 0; k < 4; k++)
            for (int l = 0; l < 4; l++)
                if (j >= 2 || k >= 2 || l >= 2) {
                    const double v = a[16 * j + 4 * k + l];
                    mx = fmax(mx, fabs(v));
                    ss = fma(v, v, ss);
                }
    return norm == GS_NORM_MAX ? mx : sqrt(ss);
}

__global__ void __launch_bounds__(128) k_estimate_f64(GsProblem P, int level, const double *__restrict__ A,
                                                      int64_t n, const uint64_t *parents, const uint8_t *vmask,
                                                      uint8_t *__restrict__ dec, double *__restrict__ bounds,
                                                      const int32_t *__restrict__ list, const unsigned *nlist)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (list) {
        // compacted list of the cubes to estimate (the rest keep DEC_INVALID)
        if (q >= (int64_t)*nlist) return;
        q = list[q];
    } else if (q >= n) {
        return;
    }
    Octet oc = octet_of(P, level, parents, vmask, q >> 3);
    if (!((oc.vmask >> (q & 7)) & 1)) { dec[q] = DEC_INVALID; return; }
    double a[64];
#pragma unroll
    for (int t = 0; t < 64; t++) a[t] = A[q * 64 + t];
    double b[6], rm, sens, rrel = 1e30;
    estimate_bounds_sens<double>(a, b, rm, sens, 0, -1, 0, nullptr, P.near ? &rrel : nullptr);
    if (P.norm != GS_NORM_SUM) b[3] = high_norm(a, P.norm);
    const int d = P.order == GS_ORDER_LITERAL ? decide_literal(b, P.c, P.precision, level, P.max_depth)
                                              : decide<double>(b, P.c, P.precision, level, P.max_depth);
    dec[q] = (uint8_t)d;
    if (P.near && b[4] != 0.0) {
        // the margins of the decision against its thresholds
        const double scale = fabs(P.c) + fabs(b[0]) + fabs(b[1]);
        if (fmin(fabs(P.c - b[0]), fabs(b[1] - P.c)) < GS_NEAR_REL * scale) atomicAdd(&P.near[0], 1ull);
        if (d != DEC_DISCARD && fabs(P.precision - b[3]) < GS_NEAR_REL * (P.precision + b[3]))
            atomicAdd(&P.near[1], 1ull);
        if (rrel < GS_NEAR_REL) atomicAdd(&P.near[2], 1ull);
    }
    if (bounds)
        for (int t = 0; t < 6; t++) bounds[q * 6 + t] = b[t];
}

// FP64 first pass (default decision order and norm, no bounds wanted):
// invalid cubes and cubes whose corner values of P~ straddle c by more than
// the rounding of those sums (1e-12 sum|A|) are decided here; the FP64 bounds
// enclose P~ up to rounding, so the SVD estimate would keep them too, and
// the precision sum is taken in the same order as there.  The rest go to a
// list for the SVD estimate.
__global__ void __launch_bounds__(256) k_estimate_pre64(GsProblem P, int level, const double *__restrict__ A, int64_t n,
                                                        const uint64_t *parents, const uint8_t *vmask,
                                                        uint8_t *__restrict__ dec, int32_t *__restrict__ list,
                                                        unsigned *nlist)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool slow = false;
    if (q < n) {
        Octet oc = octet_of(P, level, parents, vmask, q >> 3);
        if (!((oc.vmask >> (q & 7)) & 1)) {
            dec[q] = DEC_INVALID;
        } else {
            double a[64];
            double tot = 0.0, high = 0.0;
#pragma unroll
            for (int t = 0; t < 64; t++) {
                a[t] = A[q * 64 + t];
                tot += fabs(a[t]);
                if ((t >> 4) >= 2 || ((t >> 2) & 3) >= 2 || (t & 3) >= 2) high += fabs(a[t]);
            }
            double lo, hi;
            corner_range<double>(a, lo, hi);
            const double cm = 1e-12 * tot;
            if (tot == 0.0) {
                // no atom reaches the cube: the full estimate discards it
                dec[q] = DEC_DISCARD;
            } else if (hi - P.c > cm && P.c - lo > cm) {
                dec[q] = (uint8_t)(high <= P.precision ? DEC_ACCEPT : (level >= P.max_depth ? DEC_FORCED : DEC_SPLIT));
                if (P.near && fabs(P.precision - high) < GS_NEAR_REL * (P.precision + high))
                    atomicAdd(&P.near[1], 1ull);
            } else {
                slow = true;
            }
        }
    }
    const unsigned bal = __ballot_sync(0xffffffffu, slow);
    if (!bal) return;
    const unsigned lane = threadIdx.x & 31;
    unsigned wb = 0;
    if (lane == 0) wb = atomicAdd(nlist, (unsigned)__popc(bal));
    wb = __shfl_sync(0xffffffffu, wb, 0);
    if (slow) list[wb + __popc(bal & ((1u << lane) - 1u))] = (int32_t)q;
}

int gs_estimate_f64(const GsProblem &P, int level, const double *d_A, int64_t n_cubes, const uint64_t *d_parents,
                    const uint8_t *d_vmask, uint8_t *d_dec, double *d_bounds, cudaStream_t st)
{
    if (n_cubes <= 0) return GS_OK;
    if (!d_bounds && P.order == GS_ORDER_BOUNDS_FIRST && P.norm == GS_NORM_SUM && n_cubes < ((int64_t)1 << 31)) {
        int32_t *list = nullptr;
        unsigned *nlist = nullptr;
        int rc = gs_alloc((void **)&list, sizeof(int32_t) * (size_t)n_cubes, st);
        if (!rc) rc = gs_alloc((void **)&nlist, sizeof(unsigned), st);
        if (rc) { gs_free(list, st); return rc; }
        GS_CHECK(cudaMemsetAsync(nlist, 0, sizeof(unsigned), st));
        GS_LAUNCH(k_estimate_pre64, (unsigned)((n_cubes + 255) / 256), 256, 0, st)(P, level, d_A, n_cubes, d_parents,
                                                                                d_vmask, d_dec, list, nlist);
        GS_LAUNCH(k_estimate_f64, (unsigned)((n_cubes + 127) / 128), 128, 0, st)(P, level, d_A, n_cubes, d_parents,
                                                                         d_vmask, d_dec, nullptr, list, nlist);
        gs_free(list, st);
        gs_free(nlist, st);
        GS_CHECK(cudaGetLastError());
        return GS_OK;
    }
    GS_LAUNCH(k_estimate_f64, (unsigned)((n_cubes + 127) / 128), 128, 0, st)(P, level, d_A, n_cubes, d_parents, d_vmask,
                                                                     d_dec, d_bounds, nullptr, nullptr);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// ---------------------------------------------------------------- re-expansion
// child tensors from the parents' (one thread per child): the parent's
// polynomial re-expanded on the child box, axis by axis
__global__ void k_reexpand(const double *__restrict__ Apar, int64_t n_oct, double *__restrict__ A_out)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_oct * 8) return;
    const int c = (int)(t & 7), hx = c & 1, hy = (c >> 1) & 1, hz = c >> 2;
    const double *P = Apar + (t >> 3) * 64;
    double B[64], C[64];
    // along x (first index)
    for (int p = 0; p < 4; p++)
        for (int kl = 0; kl < 16; kl++) {
            double acc = 0.0;
            for (int j = 0; j < 4; j++) acc = fma(c_reexp[hx][p][j], P[16 * j + kl], acc);
            B[16 * p + kl] = acc;
        }
    // along y
    for (int p = 0; p < 4; p++)
        for (int q = 0; q < 4; q++)
            for (int l = 0; l < 4; l++) {
                double acc = 0.0;
                for (int k = 0; k < 4; k++) acc = fma(c_reexp[hy][q][k], B[16 * p + 4 * k + l], acc);
                C[16 * p + 4 * q + l] = acc;
            }
    // along z
    double *out = A_out + t * 64;
    for (int pq = 0; pq < 16; pq++)
        for (int r = 0; r < 4; r++) {
            double acc = 0.0;
            for (int l = 0; l < 4; l++) acc = fma(c_reexp[hz][r][l], C[4 * pq + l], acc);
            out[4 * pq + r] = acc;
        }
}

int gs_reexpand(const double *d_Apar, int64_t n_oct, double *d_A, cudaStream_t st)
{
    if (n_oct <= 0) return GS_OK;
    GS_LAUNCH(k_reexpand, (unsigned)((n_oct * 8 + 127) / 128), 128, 0, st)(d_Apar, n_oct, d_A);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// tensors of the split cubes, in the order of the next level's parents
__global__ void k_split_tensors(const uint8_t *__restrict__ dec, int64_t n, const int64_t *__restrict__ off,
                                const double *__restrict__ A, double *__restrict__ Anext)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 64) return;
    const int64_t q = t >> 6;
    if (dec[q] != DEC_SPLIT) return;
    Anext[(off[q] & 0xffffffffll) * 64 + (t & 63)] = A[t];
}

// ---------------------------------------------------------------- compaction
// packed[q] = [SPLIT] + [ACCEPT or FORCED] << 32; after an exclusive scan the
// low half is the cube's slot among the next level's parents, the high half
// its slot among the accepted cubes.  counters: examined, discarded,
// accepted, forced, split.
__global__ void __launch_bounds__(256) k_level_count(const uint8_t *__restrict__ dec, int64_t n,
                                                     int64_t *__restrict__ packed, unsigned long long *counters)
{
    // grid-stride; counts kept per thread and reduced once per block, so the
    // five global counters see one atomic per block
    unsigned cnt[5] = {0, 0, 0, 0, 0};
    for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < n; q += (int64_t)gridDim.x * blockDim.x) {
        unsigned d = dec[q];
        packed[q] = (int64_t)(d == DEC_SPLIT) | ((int64_t)(d == DEC_ACCEPT || d == DEC_FORCED) << 32);
        cnt[0] += d != DEC_INVALID;
        cnt[1] += d == DEC_DISCARD;
        cnt[2] += d == DEC_ACCEPT;
        cnt[3] += d == DEC_FORCED;
        cnt[4] += d == DEC_SPLIT;
    }
    __shared__ unsigned long long sh[5];
    if (threadIdx.x < 5) sh[threadIdx.x] = 0;
    __syncthreads();
    for (int k = 0; k < 5; k++) {
        unsigned v = cnt[k];
        for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
        if ((threadIdx.x & 31) == 0 && v) atomicAdd(&sh[k], (unsigned long long)v);
    }
    __syncthreads();
    if (threadIdx.x < 5 && sh[threadIdx.x]) atomicAdd(&counters[threadIdx.x], sh[threadIdx.x]);
}

// mol (nullable, the batched form): the octets' molecules, passed on to the
// children (next_mol) and the accepted cubes (acc_mol)
__global__ void k_level_emit(GsProblem P, int level, const uint64_t *parents, const uint8_t *vmask,
                             const uint8_t *__restrict__ dec, int64_t n, const int64_t *__restrict__ off,
                             uint64_t *__restrict__ next, uint64_t *__restrict__ acc, const int32_t *__restrict__ mol,
                             int32_t *__restrict__ next_mol, int32_t *__restrict__ acc_mol)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    unsigned d = dec[q];
    if (d != DEC_SPLIT && d != DEC_ACCEPT && d != DEC_FORCED) return;
    Octet oc = octet_of(P, level, parents, vmask, q >> 3);
    int c = (int)(q & 7);
    uint64_t key = gk_make(2 * oc.I + (c & 1), 2 * oc.J + ((c >> 1) & 1), 2 * oc.K + (c >> 2), GT_CUBE, (unsigned)level);
    int64_t o = off[q];
    if (d == DEC_SPLIT) {
        next[o & 0xffffffffll] = key;
        if (mol) next_mol[o & 0xffffffffll] = mol[q >> 3];
    } else {
        acc[o >> 32] = key;
        if (mol) acc_mol[o >> 32] = mol[q >> 3];
    }
}

int gs_level_compact(const GsProblem &P, int level, const uint64_t *d_parents, const uint8_t *d_vmask, int64_t n_oct,
                     const uint8_t *d_dec, uint64_t **d_next, int64_t *n_next, uint64_t *d_acc_base,
                     int64_t acc_cap, int64_t *n_acc, unsigned long long *d_counters, cudaStream_t st,
                     const double *d_A, double **d_nextA, const int32_t *d_mol, int32_t **d_next_mol,
                     int32_t *d_acc_mol)
{
    if (d_nextA) *d_nextA = nullptr;
    if (d_next_mol) *d_next_mol = nullptr;
    int64_t n = n_oct * 8;
    *d_next = nullptr; *n_next = 0; *n_acc = 0;
    if (n <= 0) return GS_OK;
    int64_t *packed = nullptr, *tot = nullptr;
    int rc = gs_alloc((void **)&packed, sizeof(int64_t) * (size_t)(n + 1), st);
    if (!rc) rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
    if (rc) { gs_free(packed, st); return rc; }
    cudaMemsetAsync(packed + n, 0, sizeof(int64_t), st);
    {
        int64_t nb = (n + 255) / 256;
        GS_LAUNCH(k_level_count, (unsigned)(nb < 152 * 16 ? nb : 152 * 16), 256, 0, st)(d_dec, n, packed, d_counters);
    }
    rc = gs_scan_i64(packed, n + 1, tot, st);
    int64_t h = 0;
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(&h, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = gs_sync(st);
        if (e != cudaSuccess) rc = gs_fail_cuda(e, "level counts", __FILE__, __LINE__);
    }
    int64_t ns = h & 0xffffffffll, na = h >> 32;
    if (!rc && na > acc_cap) rc = gs_fail(GS_ERR_CAPACITY, "accepted-cube buffer too small");
    if (!rc && ns > 0) rc = gs_alloc((void **)d_next, sizeof(uint64_t) * (size_t)ns, st);
    if (!rc && ns > 0 && d_mol) rc = gs_alloc((void **)d_next_mol, sizeof(int32_t) * (size_t)ns, st);
    if (!rc) GS_LAUNCH(k_level_emit, (unsigned)((n + 255) / 256), 256, 0, st)(P, level, d_parents, d_vmask, d_dec, n, packed,
                                                                      *d_next, d_acc_base, d_mol,
                                                                      d_mol ? *d_next_mol : nullptr, d_acc_mol);
    if (!rc && d_A && d_nextA && ns > 0) {
        rc = gs_alloc((void **)d_nextA, sizeof(double) * 64 * (size_t)ns, st);
        if (!rc)
            GS_LAUNCH(k_split_tensors, (unsigned)((n * 64 + 255) / 256), 256, 0, st)(d_dec, n, packed, d_A, *d_nextA);
    }
    gs_free(packed, st); gs_free(tot, st);
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    *n_next = ns;
    *n_acc = na;
    return GS_OK;
}

// explicit keys of the root blocks (2x2x2 root cubes), x fastest
__global__ void k_root_blocks(int64_t bx, int64_t by, int64_t n, uint64_t *keys)
{
    int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    keys[o] = gk_make(o % bx, (o / bx) % by, o / (bx * by), GT_CUBE, 0);
}

int gs_root_blocks(const GsProblem &P, uint64_t **d_keys, int64_t *n, cudaStream_t st)
{
    int64_t bx = (P.nroot[0] + 1) / 2, by = (P.nroot[1] + 1) / 2, bz = (P.nroot[2] + 1) / 2;
    *n = bx * by * bz;
    int rc = gs_alloc((void **)d_keys, sizeof(uint64_t) * (size_t)*n, st);
    if (rc) return rc;
    GS_LAUNCH(k_root_blocks, (unsigned)((*n + 255) / 256), 256, 0, st)(bx, by, *n, *d_keys);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// ================================================================ mixed precision
// FP32 accumulation.  Atom centres and lattice coordinates are taken relative
// to the origin as two-float sums, so differences x - e keep ~1e-7 A; the
// 1-D factors use gs_ex2; each lane sums 8 atoms plainly and folds the batch
// into a Kahan-compensated accumulator.  Per cube it also sums
// w * Fx * Fy * Fz (F = the largest value of the atom's 1-D factor on the
// cube's interval), an upper bound of every term's size from which the
// error band of the FP32 tensor is derived.
// Per queued atom the coefficient lane writes the products the update needs:
// WXY[cy][cx][j][k] = w X_cx[j] Y_cy[k] (64), Z[cz][l] with each value twice
// (16) and, per child, w Fx Fy Fz (8); the update of lane (child, j) is then
// three 16-byte loads and 8 paired FMA (f32x2) per atom: the pairs run over
// k = (0,1) and (2,3) against (Z[l], Z[l]).  Paired operations round each
// element as the scalar ones do.  The eight lanes of a quarter warp read
// eight consecutive 16-byte words; the record stride (23 words of 16 bytes)
// spreads the coefficient lanes' stores over all banks.
#define ACF_WXY 0
#define ACF_Z 64
#define ACF_EB 80
#define ACF_STRIDE 92

// GV: quadrature variant (a compile-time constant, so the node loop unrolls
// and the nodes and weights are immediate constant-bank operands)
template <int GV, int NQ, bool BATCH>
__global__ void __launch_bounds__(32 * ACC_WARPS, 4) k_accum_f32(GsProblem P0, int level, const uint64_t *parents,
                                                                  const uint8_t *vmask, int64_t n_oct,
                                                                  float hf, int lat_exact, float *__restrict__ A_out,
                                                                  float *__restrict__ E_out,
                                                                  unsigned long long *pairs,
                                                                  unsigned long long *atom_octets,
                                                                  const GsProblem *__restrict__ probs,
                                                                  const int32_t *__restrict__ mol)
{
    unsigned long long my_pairs = 0, my_atoms = 0;
    __shared__ __align__(16) float s_cf[ACC_WARPS][32][ACF_STRIDE];
    __shared__ int s_qi[ACC_WARPS][ACC_Q];
    __shared__ uint8_t s_qm[ACC_WARPS][ACC_Q];
    const int lane = threadIdx.x & 31, wl = threadIdx.x >> 5;
    const unsigned below = (1u << lane) - 1u;
    const int c = lane >> 2, j = lane & 3;
    const int cx = c & 1, cy = (c >> 1) & 1, cz = c >> 2;
    const int oWXY = ACF_WXY + ((cy * 2 + cx) * 4 + j) * 4, oZ = ACF_Z + 8 * cz, oEB = ACF_EB + c;
    const float nDl2e = (float)(-P0.D * 1.4426950408889634);
    const float hh = 0.5f * hf;
    for (int64_t o = (int64_t)blockIdx.x * ACC_WARPS + wl; o < n_oct; o += (int64_t)gridDim.x * ACC_WARPS) {
        const GsProblem &P = BATCH ? probs[mol[o]] : P0;
        Octet q = octet_of(P, level, parents, vmask, o);
        int64_t base[3] = {2 * q.I, 2 * q.J, 2 * q.K};
        // interval ends relative to the origin as hi + lo floats; when the
        // lattice spacing has few mantissa bits the products are exact in FP32
        float eh[3][3], el[3][3];
        for (int a = 0; a < 3; a++)
            for (int t = 0; t < 3; t++) {
                if (lat_exact) {
                    // indices < 2^18: convert through int32 (64-bit conversions are slow)
                    eh[a][t] = (float)(int)(base[a] + t) * hf;
                    el[a][t] = 0.f;
                } else {
                    double rel = gs_lat(P, a, base[a] + t, level) - P.origin[a];
                    eh[a][t] = (float)rel;
                    el[a][t] = (float)(rel - (double)eh[a][t]);
                }
            }
        // [kp][l] holds the entries (k, l) = (2 kp, l) and (2 kp + 1, l);
        // ncomp is the negated Kahan compensation
        float2 acc[2][4], ncomp[2][4], part[2][4];
#pragma unroll
        for (int kp = 0; kp < 2; kp++)
#pragma unroll
            for (int l = 0; l < 4; l++) {
                acc[kp][l] = make_float2(0.f, 0.f);
                ncomp[kp][l] = make_float2(0.f, 0.f);
                part[kp][l] = make_float2(0.f, 0.f);
            }
        float eb = 0.f;
        int nb = 0, qn = 0;
        const uint8_t vm = q.vmask;

        // Kahan step y = part - comp, s = acc + y, comp = (s - acc) - y; each
        // subtraction is an FMA with -1, which rounds as the subtraction does
        auto fold = [&]() {
            const float2 m1 = make_float2(-1.f, -1.f);
#pragma unroll
            for (int kp = 0; kp < 2; kp++)
#pragma unroll
                for (int l = 0; l < 4; l++) {
                    const float2 y = __fadd2_rn(part[kp][l], ncomp[kp][l]);
                    const float2 sm = __fadd2_rn(acc[kp][l], y);
                    const float2 t = __ffma2_rn(acc[kp][l], m1, sm);
                    ncomp[kp][l] = __ffma2_rn(t, m1, y);
                    acc[kp][l] = sm;
                    part[kp][l] = make_float2(0.f, 0.f);
                }
            nb = 0;
        };

        // coefficients of the queued atoms (one lane per atom), then the
        // rank-one updates (lane = child, x index); nb and the folds are
        // warp-uniform
        auto process = [&](int nproc) {
            if (lane < nproc) {
                int i = s_qi[wl][lane];
                const float ah[3] = {P.hx[i], P.hy[i], P.hz[i]}, al[3] = {P.lx[i], P.ly[i], P.lz[i]};
                float cf[3][2][4], F[3][2];
#pragma unroll
                for (int a = 0; a < 3; a++) {
                    float d[3], f[3];
#pragma unroll
                    for (int t = 0; t < 3; t++) {
                        d[t] = (eh[a][t] - ah[a]) + (el[a][t] - al[a]);   // e_t - x
                        f[t] = gs_ex2(nDl2e * d[t] * d[t]);
                    }
#pragma unroll
                    for (int hI = 0; hI < 2; hI++) {
                        float m = d[hI] + hh;   // interval centre - x
                        float a0 = 0.f, a1 = 0.f, a2 = 0.f, a3 = 0.f;
#pragma unroll
                        for (int k = 0; k < NQ; k++) {
                            float dk = fmaf(hh, c_gq_tf[GV][k], m);
                            float fk = gs_ex2(nDl2e * dk * dk);
                            a0 = fmaf(c_gq_Wf[GV][k][0], fk, a0);
                            a1 = fmaf(c_gq_Wf[GV][k][1], fk, a1);
                            a2 = fmaf(c_gq_Wf[GV][k][2], fk, a2);
                            a3 = fmaf(c_gq_Wf[GV][k][3], fk, a3);
                        }
                        float fa = f[hI], fb = f[hI + 1];
                        float eR = fb - (a0 + a1 + a2 + a3), eL = fa - (a0 - a1 + a2 - a3);
                        cf[a][hI][0] = a0;
                        cf[a][hI][1] = a1;
                        cf[a][hI][2] = a2 + 0.5f * (eR + eL);
                        cf[a][hI][3] = a3 + 0.5f * (eR - eL);
                        bool inside = d[hI] <= 0.f && d[hI + 1] >= 0.f;
                        F[a][hI] = inside ? 1.f : fmaxf(fa, fb);
                    }
                }
                const float w = P.fw[i];
                float *rec = s_cf[wl][lane];
#pragma unroll
                for (int x = 0; x < 2; x++)
#pragma unroll
                    for (int jj = 0; jj < 4; jj++) {
                        float wx = w * cf[0][x][jj];
#pragma unroll
                        for (int y = 0; y < 2; y++) {
                            float4 v = make_float4(wx * cf[1][y][0], wx * cf[1][y][1], wx * cf[1][y][2], wx * cf[1][y][3]);
                            *reinterpret_cast<float4 *>(rec + ACF_WXY + ((y * 2 + x) * 4 + jj) * 4) = v;
                        }
                    }
#pragma unroll
                for (int z = 0; z < 2; z++) {
                    *reinterpret_cast<float4 *>(rec + ACF_Z + 8 * z) =
                        make_float4(cf[2][z][0], cf[2][z][0], cf[2][z][1], cf[2][z][1]);
                    *reinterpret_cast<float4 *>(rec + ACF_Z + 8 * z + 4) =
                        make_float4(cf[2][z][2], cf[2][z][2], cf[2][z][3], cf[2][z][3]);
                }
                float e8[8];
#pragma unroll
                for (int cc = 0; cc < 8; cc++) e8[cc] = w * F[0][cc & 1] * F[1][(cc >> 1) & 1] * F[2][cc >> 2];
                *reinterpret_cast<float4 *>(rec + ACF_EB) = make_float4(e8[0], e8[1], e8[2], e8[3]);
                *reinterpret_cast<float4 *>(rec + ACF_EB + 4) = make_float4(e8[4], e8[5], e8[6], e8[7]);
            }
            __syncwarp();
            auto upd = [&](int t) {
                const unsigned mt = s_qm[wl][t];
                const float *rec = s_cf[wl][t];
                float4 xy = *reinterpret_cast<const float4 *>(rec + oWXY);
                const float4 za = *reinterpret_cast<const float4 *>(rec + oZ);
                const float4 zb = *reinterpret_cast<const float4 *>(rec + oZ + 4);
                float e1 = rec[oEB];
                if (mt != 0xFFu && !((mt >> c) & 1u)) {
                    // this atom does not reach this lane's child
                    xy = make_float4(0.f, 0.f, 0.f, 0.f);
                    e1 = 0.f;
                }
                const float2 xk[2] = {make_float2(xy.x, xy.y), make_float2(xy.z, xy.w)};
                const float2 zl[4] = {make_float2(za.x, za.y), make_float2(za.z, za.w), make_float2(zb.x, zb.y),
                                      make_float2(zb.z, zb.w)};
#pragma unroll
                for (int kp = 0; kp < 2; kp++)
#pragma unroll
                    for (int l = 0; l < 4; l++) part[kp][l] = __ffma2_rn(xk[kp], zl[l], part[kp][l]);
                eb += e1;
            };
            int t = 0;
            for (; t + 2 <= nproc; t += 2) {
                upd(t);
                upd(t + 1);
                nb += 2;
                if (nb >= 8) fold();
            }
            if (t < nproc) {
                upd(t);
                if (++nb >= 8) fold();
            }
            __syncwarp();
        };

        // membership of one candidate per lane (i < 0: none): FP32 box
        // distance with a relative margin, the exact FP64 test inside the
        // margin; members join the atom queue
        auto filter = [&](int i) {
            unsigned m = 0;
            if (i >= 0) {
                const float ah[3] = {P.hx[i], P.hy[i], P.hz[i]}, al[3] = {P.lx[i], P.ly[i], P.lz[i]};
                float g2[3][2];
#pragma unroll
                for (int a = 0; a < 3; a++)
#pragma unroll
                    for (int hI = 0; hI < 2; hI++) {
                        float dlo = (eh[a][hI] - ah[a]) + (el[a][hI] - al[a]);
                        float dhi = (ah[a] - eh[a][hI + 1]) + (al[a] - el[a][hI + 1]);
                        float g = fmaxf(0.f, fmaxf(dlo, dhi));
                        g2[a][hI] = g * g;
                    }
                const float R2 = P.fR2[i];
                const float tol = 1e-5f * R2 + 1e-5f;
                unsigned nearm = 0;
#pragma unroll
                for (int cc = 0; cc < 8; cc++) {
                    float d2 = g2[0][cc & 1] + g2[1][(cc >> 1) & 1] + g2[2][cc >> 2];
                    if (d2 < R2 - tol) m |= 1u << cc;
                    else if (d2 <= R2 + tol) nearm |= 1u << cc;
                }
                m &= vm;
                nearm &= vm;
                // near the cutoff sphere: the exact FP64 membership test
                while (nearm) {
                    const int cc = __ffs(nearm) - 1;
                    nearm &= nearm - 1;
                    double x = P.ax[i], y = P.ay[i], z = P.az[i];
                    int64_t ix = base[0] + (cc & 1), iy = base[1] + ((cc >> 1) & 1), iz = base[2] + (cc >> 2);
                    double dx = gs_axis_gap(gs_lat(P, 0, ix, level), gs_lat(P, 0, ix + 1, level), x);
                    double dy = gs_axis_gap(gs_lat(P, 1, iy, level), gs_lat(P, 1, iy + 1, level), y);
                    double dz = gs_axis_gap(gs_lat(P, 2, iz, level), gs_lat(P, 2, iz + 1, level), z);
                    double dd = __dadd_rn(__dadd_rn(__dmul_rn(dx, dx), __dmul_rn(dy, dy)), __dmul_rn(dz, dz));
                    if (dd <= P.aR2[i]) m |= 1u << cc;
                }
            }
            my_pairs += __popc(m);
            unsigned bal = __ballot_sync(0xffffffffu, m != 0);
            if (lane == 0) my_atoms += __popc(bal);
            int pos = qn + __popc(bal & below);
            if (m) { s_qi[wl][pos] = i; s_qm[wl][pos] = (uint8_t)m; }
            qn += __popc(bal);
            __syncwarp();
            if (qn >= 32) {
                process(32);
                int rest = qn - 32;
                int mi = 0; uint8_t mm = 0;
                if (lane < rest) { mi = s_qi[wl][32 + lane]; mm = s_qm[wl][32 + lane]; }
                __syncwarp();
                if (lane < rest) { s_qi[wl][lane] = mi; s_qm[wl][lane] = mm; }
                __syncwarp();
                qn = rest;
            }
        };

        if (vm) {
            float flo[3] = {eh[0][0], eh[1][0], eh[2][0]}, fhi[3] = {eh[0][2], eh[1][2], eh[2][2]};
            gs_warp_candidates(P, flo, fhi, lane, filter);
            if (qn > 0) process(qn);
            fold();
        }
        float *dst = A_out + ((size_t)o * 8 + c) * 64 + 16 * j;
#pragma unroll
        for (int kp = 0; kp < 2; kp++) {
            float2 v[4];
#pragma unroll
            for (int l = 0; l < 4; l++) v[l] = __fadd2_rn(acc[kp][l], ncomp[kp][l]);   // acc - comp
            *reinterpret_cast<float4 *>(dst + 4 * (2 * kp)) = make_float4(v[0].x, v[1].x, v[2].x, v[3].x);
            *reinterpret_cast<float4 *>(dst + 4 * (2 * kp + 1)) = make_float4(v[0].y, v[1].y, v[2].y, v[3].y);
        }
        if (j == 0) E_out[(size_t)o * 8 + c] = eb;
    }
    if (pairs) {
        for (int off = 16; off > 0; off >>= 1) my_pairs += __shfl_xor_sync(0xffffffffu, my_pairs, off);
        if (lane == 0 && my_pairs) atomicAdd(pairs, my_pairs);
    }
    if (atom_octets && lane == 0 && my_atoms) atomicAdd(atom_octets, my_atoms);
}

int gs_accum_f32(const GsProblem &P, int level, const uint64_t *d_parents, const uint8_t *d_vmask, int64_t n_oct,
                 float *d_A, float *d_err, unsigned long long *d_pairs, unsigned *d_status, cudaStream_t st, float *ms,
                 unsigned long long *d_atom_octets, const GsProblem *d_probs, const int32_t *d_mol)
{
    if (n_oct <= 0) return GS_OK;
    double h = gs_h(P, level);
    int gv = gq_variant(P.D, 0.5 * h, true);
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    if (ms) { cudaEventCreate(&e0); cudaEventCreate(&e1); cudaEventRecord(e0, st); }
    // grid shapes the tuner chooses from: up to 64, 16 or 4 blocks per SM
    // (each warp takes every grid-th octet; the sums do not depend on it)
    static const int64_t caps[3] = {152 * 64, 152 * 16, 152 * 4};
    auto run = [&](int shape, unsigned long long *scratch) {
        int64_t g = (n_oct + ACC_WARPS - 1) / ACC_WARPS;
        if (g > caps[shape]) g = caps[shape];
        const unsigned grid = (unsigned)(g < 1 ? 1 : g);
        unsigned long long *pairs = scratch ? scratch : d_pairs;
        unsigned long long *aoct = scratch ? (d_atom_octets ? scratch + 1 : nullptr) : d_atom_octets;
#define GS_ACC32(V, N)                                                                                              \
    do {                                                                                                            \
        if (d_probs)                                                                                                \
            GS_LAUNCH((k_accum_f32<V, N, true>), grid, 32 * ACC_WARPS, 0, st)(P, level, d_parents, d_vmask, n_oct,  \
                                                                             (float)h, P.lat_exact_f32, d_A, d_err, \
                                                                             pairs, aoct, d_probs, d_mol);          \
        else                                                                                                        \
            GS_LAUNCH((k_accum_f32<V, N, false>), grid, 32 * ACC_WARPS, 0, st)(P, level, d_parents, d_vmask, n_oct, \
                                                                              (float)h, P.lat_exact_f32, d_A,      \
                                                                              d_err, pairs, aoct, nullptr, nullptr); \
    } while (0)
        switch (gv) {
        case 5: GS_ACC32(5, 5); break;
        case 4: GS_ACC32(4, 6); break;
        case 0: GS_ACC32(0, 8); break;
        case 1: GS_ACC32(1, 12); break;
        default: GS_ACC32(2, 16); break;
        }
#undef GS_ACC32
    };
    char name[32];
    snprintf(name, sizeof(name), "k_accum_f32<%d>", gv);
    int rc = gs_tune_run(name, n_oct, 3, st, run);
    if (rc) {
        if (ms) { cudaEventDestroy(e0); cudaEventDestroy(e1); }
        return rc;
    }
    if (ms) {
        cudaEventRecord(e1, st);
        cudaEventSynchronize(e1);
        float t = 0;
        cudaEventElapsedTime(&t, e0, e1);
        *ms += t;
        cudaEventDestroy(e0); cudaEventDestroy(e1);
    }
    (void)d_status;
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// FP32 estimate.  A decision is final when every margin it rests on exceeds
// the band the FP32 error of A and the FP32 estimate can move it by:
//   entry error      dA = MIXED_KAPPA * E + 1e-7 sum|A|   (E = sum w Fx Fy Fz;
//                    the largest observed |A32 - A64| / E is 7.7e-7)
//   bounds L, U      4 (dA + 1e-7 sum|A|)(1 + s), s = sigma_1 over the smallest
//                    gap between kept and neighbouring singular values (the
//                    singular vectors' sensitivity); about 9x the largest
//                    change observed between the FP32 and FP64 estimates
//   rank rules       a rule within 32 dA of its 99% threshold may flip and
//                    move terms between the main part and R; the decision is
//                    final when its margin also exceeds RANK_FLIP_ALLOW times
//                    the sum of the singular values; otherwise one such rule
//                    is settled by re-estimating under the flipped rank, more
//                    by FP64
//   precision sum    |d sum|high|| <= 64 dA + rounding (kept cubes only)
// Otherwise the cube is flagged and its octet is re-evaluated in FP64.  The
// debug mode (GS debug bit 0) re-runs every cube in FP64 and counts
// disagreements; the tests require zero.
#define MIXED_KAPPA 1.5e-6f

// Largest change of L or U, relative to the sum of the outer singular values
// S, when rank rules near their 99% thresholds flip.  A flipping rule moves
// terms whose singular values sum to at most ~1% of S (the rule sits at the
// threshold); per unit of singular value, a term adds at most 16 to the
// product bound (|u| <= sum|u_a| <= 2, sum d_k <= 2, |w z| <= 4) and at most 8
// to sum|R|.  Outer rules move <= 16 (0.011 S); inner rules of term i move
// <= 8 (0.011 sigma_i) sum_k d_k <= 16 (0.011 sigma_i), <= 16 (0.011 S) over
// all terms; together <= 0.36 S.
#define RANK_FLIP_ALLOW 0.4f

// one cube's 64 coefficients (256 B, 16-byte aligned) in 16-byte loads
__device__ __forceinline__ void load_tensor_f32(const float *__restrict__ src, float *a)
{
    const float4 *s4 = reinterpret_cast<const float4 *>(src);
#pragma unroll
    for (int t = 0; t < 16; t++) {
        const float4 v = __ldg(s4 + t);
        a[4 * t] = v.x; a[4 * t + 1] = v.y; a[4 * t + 2] = v.z; a[4 * t + 3] = v.w;
    }
}


// Cubes whose corner values of P~ straddle c by more than the FP32 error of
// those sums are kept by the FP64 estimate whatever its SVD gives: L <= min P~
// and max P~ <= U hold for any factorisation, since R = A - A~ is taken
// exactly and the 1-D and product bounds are enclosures.  Their decision needs
// only the precision sum.  Returns false for the cubes that need the bounds.
__device__ __forceinline__ bool estimate_fast_f32(const GsProblem &P, int level, const float *__restrict__ A,
                                                  const float *__restrict__ E, int64_t q, const uint64_t *parents,
                                                  const uint8_t *vmask, uint8_t *__restrict__ dec,
                                                  uint8_t *__restrict__ flag, unsigned long long *why_cnt,
                                                  float *__restrict__ dbg)
{
    Octet oc = octet_of(P, level, parents, vmask, q >> 3);
    if (!((oc.vmask >> (q & 7)) & 1)) { dec[q] = DEC_INVALID; flag[q] = 0; return true; }
    float a[64];
    load_tensor_f32(A + q * 64, a);
    float tot = 0.f, high = 0.f;
#pragma unroll
    for (int t = 0; t < 64; t++) {
        tot += fabsf(a[t]);
        if ((t >> 4) >= 2 || ((t >> 2) & 3) >= 2 || (t & 3) >= 2) high += fabsf(a[t]);
    }
    if (tot == 0.f && E[q] == 0.f) {
        // no atom reaches the cube: P~ = 0 and the full estimate discards it
        // (zero bounds, no flag); common among the root cubes
        dec[q] = DEC_DISCARD;
        flag[q] = 0;
        if (why_cnt) atomicAdd(&why_cnt[10], 1ull);   // decided without the SVD
        if (dbg) {
            float *o = dbg + 6 * q;
            o[0] = o[1] = o[2] = o[3] = o[4] = 0.f;
            o[5] = 2.f;   // no SVD bounds: the band check skips the cube
        }
        return true;
    }
    const float c = (float)P.c, prec = (float)P.precision;
    const float dA = MIXED_KAPPA * E[q] + 1e-7f * tot;
    float lo, hi;
    corner_range<float>(a, lo, hi);
    // each corner sum moves by at most sum|dA_t| <= 64 dA, plus its own FP32
    // rounding (6 additions deep, < 4e-7 sum|A|)
    const float cm = 64.f * dA + 4e-6f * tot;
    if (!(hi - c > cm && c - lo > cm)) return false;
    const int d = high <= prec ? DEC_ACCEPT : (level >= P.max_depth ? DEC_FORCED : DEC_SPLIT);
    if (why_cnt) atomicAdd(&why_cnt[10], 1ull);   // decided without the SVD
    const bool f = level < P.max_depth && fabsf(prec - high) <= 64.f * dA + 1e-6f * high + 1e-7f * tot;
    if (f && why_cnt) atomicAdd(&why_cnt[1], 1ull);
    if (dbg) {
        float *o = dbg + 6 * q;
        o[0] = lo; o[1] = hi; o[2] = 0.f; o[3] = dA; o[4] = tot;
        o[5] = 2.f;   // no SVD bounds: the band check skips the cube
    }
    dec[q] = (uint8_t)d;
    flag[q] = f ? 1 : 0;
    return true;
}

// the full FP32 estimate of one valid cube: two-level SVD bounds, rank rules
// and the bands below
__device__ __forceinline__ void estimate_full_f32(const GsProblem &P, int level, const float *__restrict__ A,
                                                  const float *__restrict__ E, int64_t q, uint8_t *__restrict__ dec,
                                                  uint8_t *__restrict__ flag, unsigned long long *why_cnt,
                                                  float *__restrict__ dbg)
{
    float a[64];
    load_tensor_f32(A + q * 64, a);
    float tot = 0.f;
#pragma unroll
    for (int t = 0; t < 64; t++) tot += fabsf(a[t]);
    float b[6], rm;
    float sens;
    RankNear<float> rn;
    rn.m1 = rn.m2 = 1e30f; rn.who = -1; rn.alt = 0; rn.ssum = 0.f;
    estimate_bounds_sens<float>(a, b, rm, sens, 0, -1, 0, &rn);
    const float c = (float)P.c, prec = (float)P.precision;
    int d = decide<float>(b, c, prec, level, P.max_depth);
    float dA = MIXED_KAPPA * E[q] + 1e-7f * tot;
    bool f = false;
    int why = 0, alt = 0;
    if (tot > 0.f) {
        // calibrated: the largest |dL|, |dU| seen between the FP32 and FP64
        // estimates (debug mode, chain and globular molecules) is 0.85 of
        // (dA + 1e-7 sum|A|)(1 + s); the band takes 4 of it
        const float bBase = 4.f * (dA + 1e-7f * tot) * (1.f + fminf(sens, 1e4f));
        float mc = fminf(fabsf(c - b[0]), fabsf(b[1] - c));
        bool keep = b[0] <= c && c <= b[1];
        const float near = 32.f * dA + 1e-5f * tot;
        if (mc <= bBase) {
            f = true;
            why = 1;
        } else if (rn.m1 <= near && mc > bBase + RANK_FLIP_ALLOW * rn.ssum) {
            // rank rules within their band may flip, but no flip can move L
            // or U across c (see RANK_FLIP_ALLOW)
        } else if (rn.m1 <= near) {
            // a rank rule within its band may flip.  With one such rule the
            // cube is re-estimated under the flipped rank (k_estimate_alt);
            // with more, FP64 decides.
            if (rn.m2 > near && rn.alt > 0) {
                alt = 0x80 | ((rn.who + 1) << 3) | rn.alt;
            } else {
                f = true;
                why = 1;
                if (why_cnt) atomicAdd(&why_cnt[5], 1ull);   // flagged through a rank rule
            }
        }
        if (!f && keep && level < P.max_depth && fabsf(prec - b[3]) <= 64.f * dA + 1e-6f * b[3] + 1e-7f * tot) {
            f = true;
            why = 2;
        }
        if (f) alt = 0;
    } else if (E[q] > 0.f) {
        f = true;  // an all-zero FP32 tensor with contributing atoms: let FP64 decide
        why = 3;
    }
    if (why && why_cnt) atomicAdd(&why_cnt[why - 1], 1ull);
    if (dbg) {
        float *o = dbg + 6 * q;
        o[0] = b[0]; o[1] = b[1]; o[2] = sens; o[3] = dA; o[4] = tot;
        o[5] = (tot > 0.f && rn.m1 <= 32.f * dA + 1e-5f * tot) ? 1.f : 0.f;
    }
    dec[q] = (uint8_t)d;
    flag[q] = f ? 1 : (uint8_t)alt;}

// first pass: invalid and straddling cubes are decided here (one light thread
// per cube); the others go to a list that the SVD estimate runs over in full
// warps
__global__ void __launch_bounds__(256) k_estimate_pre(GsProblem P, int level, const float *__restrict__ A,
                                                      const float *__restrict__ E, int64_t n, const uint64_t *parents,
                                                      const uint8_t *vmask, uint8_t *__restrict__ dec,
                                                      uint8_t *__restrict__ flag, unsigned long long *why_cnt,
                                                      float *__restrict__ dbg, int32_t *__restrict__ list,
                                                      unsigned *nlist)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool slow = q < n && !estimate_fast_f32(P, level, A, E, q, parents, vmask, dec, flag, why_cnt, dbg);
    const unsigned bal = __ballot_sync(0xffffffffu, slow);
    if (!bal) return;
    const unsigned lane = threadIdx.x & 31;
    unsigned wb = 0;
    if (lane == 0) wb = atomicAdd(nlist, (unsigned)__popc(bal));
    wb = __shfl_sync(0xffffffffu, wb, 0);
    if (slow) list[wb + __popc(bal & ((1u << lane) - 1u))] = (int32_t)q;
}

// MINB: blocks per SM the register allocation is held to (0: none; 3 caps
// the registers at 168 and spills the rest to local memory), a shape the
// tuner chooses; the arithmetic is the same
template <int MINB>
__global__ void __launch_bounds__(128, MINB) k_estimate_f32(GsProblem P, int level, const float *__restrict__ A,
                                                            const float *__restrict__ E, uint8_t *__restrict__ dec,
                                                            uint8_t *__restrict__ flag, unsigned long long *why_cnt,
                                                            float *__restrict__ dbg, const int32_t *__restrict__ list,
                                                            const unsigned *nlist)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)*nlist) return;
    estimate_full_f32(P, level, A, E, (int64_t)list[t], dec, flag, why_cnt, dbg);
}

// cubes whose FP32 decision rests on one rank rule near its threshold
// (flag 0x80 | (rule + 1) << 3 | flipped rank) -> a compact list
__global__ void k_alt_list(const uint8_t *flag, int64_t n, int32_t *list, unsigned *nlist)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool on = q < n && (flag[q] & 0x80);
    unsigned bal = __ballot_sync(0xffffffffu, on);
    if (!bal) return;
    unsigned lane = threadIdx.x & 31, base = 0;
    if (lane == 0) base = atomicAdd(nlist, (unsigned)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (on) list[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)q;
}

// the listed cubes re-estimated under the flipped rank: the decision stands
// (flag 0) when it is the same with a margin outside the band and no other
// rule of the flipped estimate is near its threshold; otherwise FP64 decides
__global__ void __launch_bounds__(128) k_estimate_alt(GsProblem P, int level, const float *__restrict__ A,
                                                      const float *__restrict__ E, const int32_t *__restrict__ list,
                                                      const unsigned *nlist, const uint8_t *__restrict__ dec,
                                                      uint8_t *__restrict__ flag, unsigned long long *why_cnt)
{
    const int64_t nl = (int64_t)*nlist;
    for (int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; t < nl; t += (int64_t)gridDim.x * blockDim.x) {
    int64_t q = list[t];
    const unsigned code = flag[q];
    const int who = (int)((code >> 3) & 7u) - 1, altr = (int)(code & 7u);
    float a[64];
    float tot = 0.f;
#pragma unroll
    for (int k = 0; k < 64; k++) { a[k] = A[q * 64 + k]; tot += fabsf(a[k]); }
    const float c = (float)P.c, prec = (float)P.precision;
    const float dA = MIXED_KAPPA * E[q] + 1e-7f * tot;
    float b2[6], rm2, sens2;
    estimate_bounds_sens<float>(a, b2, rm2, sens2, who < 0 ? altr : 0, who, who < 0 ? 0 : altr, nullptr);
    const float bAlt = 4.f * (dA + 1e-7f * tot) * (1.f + fminf(sens2, 1e4f));
    const float mc2 = fminf(fabsf(c - b2[0]), fabsf(b2[1] - c));
    const bool ok = rm2 > 32.f * dA + 1e-5f * tot && decide<float>(b2, c, prec, level, P.max_depth) == (int)dec[q] &&
                    mc2 > bAlt;
    flag[q] = ok ? 0 : 1;
    if (!ok && why_cnt) {
        atomicAdd(&why_cnt[0], 1ull);
        atomicAdd(&why_cnt[5], 1ull);
    }
    }
}

int gs_estimate_f32(const GsProblem &P, int level, const float *d_A, const float *d_err, int64_t n_cubes,
                    const uint64_t *d_parents, const uint8_t *d_vmask, uint8_t *d_dec, uint8_t *d_flag,
                    cudaStream_t st, unsigned long long *d_why, float *d_dbg)
{
    if (n_cubes <= 0) return GS_OK;
    int32_t *list = nullptr;
    unsigned *nlist = nullptr;
    int rc = gs_alloc((void **)&list, sizeof(int32_t) * (size_t)n_cubes, st);
    if (!rc) rc = gs_alloc((void **)&nlist, sizeof(unsigned), st);
    if (rc) { gs_free(list, st); return rc; }
    GS_CHECK(cudaMemsetAsync(nlist, 0, sizeof(unsigned), st));
    GS_LAUNCH(k_estimate_pre, (unsigned)((n_cubes + 255) / 256), 256, 0, st)(P, level, d_A, d_err, n_cubes, d_parents,
                                                                            d_vmask, d_dec, d_flag, d_why, d_dbg,
                                                                            list, nlist);
    const unsigned grid = (unsigned)((n_cubes + 127) / 128);
    rc = gs_tune_run("k_estimate_f32", n_cubes, 2, st, [&](int shape, unsigned long long *scratch) {
        unsigned long long *why = scratch ? (d_why ? scratch : nullptr) : d_why;
        if (shape == 0)
            GS_LAUNCH(k_estimate_f32<0>, grid, 128, 0, st)(P, level, d_A, d_err, d_dec, d_flag, why, d_dbg, list, nlist);
        else
            GS_LAUNCH(k_estimate_f32<3>, grid, 128, 0, st)(P, level, d_A, d_err, d_dec, d_flag, why, d_dbg, list, nlist);
    });
    gs_free(list, st);
    gs_free(nlist, st);
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}
__global__ void k_add_u64(unsigned long long *dst, const unsigned long long *v) { *dst += *v; }

// octets with a flagged child -> list of octet indices; counts flagged children
__global__ void k_octet_flags(const uint8_t *flag, int64_t n_oct, int64_t *cnt, unsigned long long *nflagged)
{
    int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_oct) return;
    uint64_t w = *(const uint64_t *)(flag + 8 * o);
    cnt[o] = w != 0;
    if (w && nflagged) {
        int k = 0;
        for (int c = 0; c < 8; c++) k += ((w >> (8 * c)) & 0xff) != 0;
        atomicAdd(nflagged, (unsigned long long)k);
    }
}
__global__ void k_octet_gather(const int64_t *off, int64_t n_oct, const uint64_t *parents, const uint8_t *flag,
                               uint64_t *sub_par, int64_t *sub_idx, uint8_t *sub_mask)
{
    int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n_oct || off[o + 1] == off[o]) return;
    sub_par[off[o]] = parents[o];
    sub_idx[off[o]] = o;
    uint8_t m = 0;
    for (int c = 0; c < 8; c++)
        if (flag[8 * o + c]) m |= (uint8_t)(1u << c);
    sub_mask[off[o]] = m;
}
// flagged children of the re-evaluated octets -> a compact list (any order:
// each entry is estimated on its own), so the FP64 estimate runs full warps
__global__ void k_child_list(const uint8_t *sub_mask, int64_t n_sub, int32_t *list, unsigned *nlist)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    bool on = t < n_sub * 8 && ((sub_mask[t >> 3] >> (t & 7)) & 1);
    unsigned bal = __ballot_sync(0xffffffffu, on);
    if (!bal) return;
    unsigned lane = threadIdx.x & 31, base = 0;
    if (lane == 0) base = atomicAdd(nlist, (unsigned)__popc(bal));
    base = __shfl_sync(0xffffffffu, base, 0);
    if (on) list[base + __popc(bal & ((1u << lane) - 1u))] = (int32_t)t;
}
// the FP64 decisions replace the flagged children's FP32 ones
__global__ void k_octet_scatter(const uint8_t *sub_dec, const int64_t *sub_idx, const uint8_t *sub_mask, int64_t n_sub,
                                uint8_t *dec)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n_sub * 8) return;
    if (!((sub_mask[t >> 3] >> (t & 7)) & 1)) return;
    dec[sub_idx[t >> 3] * 8 + (t & 7)] = sub_dec[t];
}
// debug: largest change of L or U between the FP32 and FP64 estimates,
// relative to (dA + 1e-7 sum|A|)(1 + s), over cubes whose rank rules are not
// within their band (those get the rank-flip allowance instead)
__global__ void k_band_ratio(const float *dbg, const double *b64, const uint8_t *d64, int64_t n, unsigned *maxbits)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n || d64[q] == DEC_INVALID) return;
    const float *o = dbg + 6 * q;
    if (o[4] <= 0.f || o[5] != 0.f) return;
    double dl = fabs((double)o[0] - b64[6 * q]), du = fabs((double)o[1] - b64[6 * q + 1]);
    double den = ((double)o[3] + 1e-7 * (double)o[4]) * (1.0 + (double)o[2]);
    float r = (float)(fmax(dl, du) / den);
    atomicMax(maxbits, __float_as_uint(r));
}

// debug: largest |A32 - A64| / E over a chunk, as float bits (non-negative)
__global__ void k_err_ratio(const float *A32, const float *E, const double *A64, int64_t n, unsigned *maxbits)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    double mx = 0;
    for (int t = 0; t < 64; t++) mx = fmax(mx, fabs((double)A32[q * 64 + t] - A64[q * 64 + t]));
    float e = E[q];
    if (e > 0.f) {
        float r = (float)(mx / e);
        atomicMax(maxbits, __float_as_uint(r));
    }
}

__global__ void k_count_mismatch(const uint8_t *a, const uint8_t *b, int64_t n, unsigned long long *mism)
{
    int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    // cube sets depend on discard / keep and split / accept; accepted vs forced is bookkeeping
    unsigned x = a[q], y = b[q];
    if (x == DEC_FORCED) x = DEC_ACCEPT;
    if (y == DEC_FORCED) y = DEC_ACCEPT;
    if (x != y) atomicAdd(mism, 1ull);
}

// one chunk of a level in mixed precision; dec receives the final decisions
// d_why: [0..2] flag reasons (bounds band, precision band, zero tensor), [3] low 32 bits = float bits of
// the largest |A32 - A64| / E seen in debug mode, [4] the same for the band ratio, [5] flags through a rank
// rule, [10] cubes decided without the SVD (corner values straddle c)
__global__ void k_gather_mol(const int64_t *__restrict__ si, int64_t m, const int32_t *__restrict__ mol,
                             int32_t *__restrict__ sub_mol)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t < m) sub_mol[t] = mol[si[t]];
}

int gs_level_mixed(const GsProblem &P, int level, const uint64_t *d_parents, int64_t n_oct, uint8_t *d_dec,
                   unsigned long long *d_pairs, unsigned long long *d_rechecked, unsigned long long *d_mism,
                   bool both, unsigned *d_status, cudaStream_t st, float *ms, unsigned long long *d_why,
                   const GsProblem *d_probs, const int32_t *d_mol, const uint8_t *d_vmask)
{
    float *A = nullptr, *E = nullptr;
    uint8_t *flag = nullptr;
    int rc = gs_alloc((void **)&A, sizeof(float) * 64 * 8 * (size_t)n_oct, st);
    if (!rc) rc = gs_alloc((void **)&E, sizeof(float) * 8 * (size_t)n_oct, st);
    if (!rc) rc = gs_alloc((void **)&flag, 8 * (size_t)n_oct, st);
    float *dbg = nullptr;
    if (!rc && both) rc = gs_alloc((void **)&dbg, sizeof(float) * 6 * 8 * (size_t)n_oct, st);
    // the counter block holds the atom-octet count 16 slots after the pair count
    if (!rc)
        rc = gs_accum_f32(P, level, d_parents, d_vmask, n_oct, A, E, d_pairs, d_status, st, ms, d_pairs + 16, d_probs,
                          d_mol);
    if (!rc) rc = gs_estimate_f32(P, level, A, E, n_oct * 8, d_parents, d_vmask, d_dec, flag, st, d_why, dbg);
    if (!rc) {
        // decisions resting on one rank rule near its threshold
        int32_t *lst = nullptr;
        unsigned *nl = nullptr;
        rc = gs_alloc((void **)&lst, sizeof(int32_t) * 8 * (size_t)n_oct, st);
        if (!rc) rc = gs_alloc((void **)&nl, sizeof(unsigned), st);
        if (!rc) {
            unsigned nb = (unsigned)((n_oct * 8 + 127) / 128);
            cudaMemsetAsync(nl, 0, sizeof(unsigned), st);
            GS_LAUNCH(k_alt_list, nb, 128, 0, st)(flag, n_oct * 8, lst, nl);
            GS_LAUNCH(k_estimate_alt, 152 * 4, 128, 0, st)(P, level, A, E, lst, nl, d_dec, flag, d_why);
        }
        gs_free(lst, st); gs_free(nl, st);
    }
    // flagged octets -> FP64
    int64_t *cnt = nullptr, *tot = nullptr;
    if (!rc) rc = gs_alloc((void **)&cnt, sizeof(int64_t) * (size_t)(n_oct + 1), st);
    if (!rc) rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
    if (!rc) {
        cudaMemsetAsync(cnt + n_oct, 0, sizeof(int64_t), st);
        GS_LAUNCH(k_octet_flags, (unsigned)((n_oct + 255) / 256), 256, 0, st)(flag, n_oct, cnt, d_rechecked);
        rc = gs_scan_i64(cnt, n_oct + 1, tot, st);
    }
    int64_t nsub = 0;
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(&nsub, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = gs_sync(st);
        if (e != cudaSuccess) rc = gs_fail_cuda(e, "recheck count", __FILE__, __LINE__);
    }
    if (!rc && nsub > 0) {
        uint64_t *sp = nullptr;
        int64_t *si = nullptr;
        double *A64 = nullptr;
        uint8_t *sd = nullptr, *sm = nullptr;
        rc = gs_alloc((void **)&sp, sizeof(uint64_t) * (size_t)nsub, st);
        if (!rc) rc = gs_alloc((void **)&si, sizeof(int64_t) * (size_t)nsub, st);
        if (!rc) rc = gs_alloc((void **)&sm, (size_t)nsub, st);
        if (!rc) rc = gs_alloc((void **)&A64, sizeof(double) * 64 * 8 * (size_t)nsub, st);
        if (!rc) rc = gs_alloc((void **)&sd, 8 * (size_t)nsub, st);
        int32_t *smol = nullptr;
        if (!rc && d_mol) rc = gs_alloc((void **)&smol, sizeof(int32_t) * (size_t)nsub, st);
        if (!rc) {
            GS_LAUNCH(k_octet_gather, (unsigned)((n_oct + 255) / 256), 256, 0, st)(cnt, n_oct, d_parents, flag, sp, si,
                                                                                  sm);
            if (d_mol) GS_LAUNCH(k_gather_mol, (unsigned)((nsub + 255) / 256), 256, 0, st)(si, nsub, d_mol, smol);
            // only the flagged children are accumulated and estimated in FP64
            rc = gs_accum_f64(P, level, sp, sm, nsub, A64, nullptr, d_status, st, nullptr, d_probs, smol);
        }
        int32_t *lst = nullptr;
        unsigned *nl = nullptr;
        if (!rc) rc = gs_alloc((void **)&lst, sizeof(int32_t) * 8 * (size_t)nsub, st);
        if (!rc) rc = gs_alloc((void **)&nl, sizeof(unsigned), st);
        if (!rc) {
            unsigned nb = (unsigned)((nsub * 8 + 127) / 128);
            cudaMemsetAsync(nl, 0, sizeof(unsigned), st);
            GS_LAUNCH(k_child_list, nb, 128, 0, st)(sm, nsub, lst, nl);
            GS_LAUNCH(k_estimate_f64, nb, 128, 0, st)(P, level, A64, nsub * 8, sp, sm, sd, nullptr, lst, nl);
        }
        gs_free(lst, st); gs_free(nl, st);
        if (!rc) GS_LAUNCH(k_octet_scatter, (unsigned)((nsub * 8 + 255) / 256), 256, 0, st)(sd, si, sm, nsub, d_dec);
        gs_free(sp, st); gs_free(si, st); gs_free(sm, st); gs_free(A64, st); gs_free(sd, st); gs_free(smol, st);
    }
    gs_free(cnt, st); gs_free(tot, st);
    if (!rc && both) {
        // debug: FP64 on every octet; count final decisions that disagree and
        // record the largest |A32 - A64| / E
        double *A64 = nullptr, *b64 = nullptr;
        uint8_t *d64 = nullptr;
        rc = gs_alloc((void **)&A64, sizeof(double) * 64 * 8 * (size_t)n_oct, st);
        if (!rc) rc = gs_alloc((void **)&b64, sizeof(double) * 6 * 8 * (size_t)n_oct, st);
        if (!rc) rc = gs_alloc((void **)&d64, 8 * (size_t)n_oct, st);
        if (!rc)
            rc = gs_accum_f64(P, level, d_parents, d_vmask, n_oct, A64, nullptr, d_status, st, nullptr, d_probs, d_mol);
        if (!rc) rc = gs_estimate_f64(P, level, A64, n_oct * 8, d_parents, d_vmask, d64, b64, st);
        if (!rc) {
            unsigned nb = (unsigned)((n_oct * 8 + 255) / 256);
            GS_LAUNCH(k_count_mismatch, nb, 256, 0, st)(d_dec, d64, n_oct * 8, d_mism);
            GS_LAUNCH(k_err_ratio, nb, 256, 0, st)(A, E, A64, n_oct * 8, (unsigned *)(d_why + 3));
            GS_LAUNCH(k_band_ratio, nb, 256, 0, st)(dbg, b64, d64, n_oct * 8, (unsigned *)(d_why + 4));
        }
        gs_free(A64, st); gs_free(b64, st); gs_free(d64, st);
    }
    gs_free(A, st);
    gs_free(E, st);
    gs_free(dbg, st);
    gs_free(flag, st);
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// ================================================================ batched form
// Several molecules share one level loop: the octets of all molecules sit in
// one array, molecule by molecule, with the molecule's index (its row in a
// device table of problem records) beside each octet.  Compaction is stable,
// so every level's arrays stay grouped by molecule and each molecule's
// octets keep the order a single-molecule run gives them.

// root blocks of every molecule: keys in the molecule's own lattice, the
// valid children (inside the molecule's root grid) and the molecule index.
// tab[g] = {first octet, bx, by, nroot x, nroot y, nroot z}; base[G] = total
__global__ void k_root_blocks_batch(const int64_t *__restrict__ tab, int G, int64_t n, uint64_t *__restrict__ keys,
                                    uint8_t *__restrict__ vmask, int32_t *__restrict__ mol)
{
    const int64_t o = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (o >= n) return;
    int lo = 0, hi = G - 1;   // last g with tab[g].first <= o
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (tab[6 * mid] <= o) lo = mid;
        else hi = mid - 1;
    }
    const int64_t *t = tab + 6 * lo;
    const int64_t r = o - t[0], bx = t[1], by = t[2];
    const int64_t I = r % bx, J = (r / bx) % by, K = r / (bx * by);
    uint8_t m = 0;
    for (int c = 0; c < 8; c++) {
        const int64_t x = 2 * I + (c & 1), y = 2 * J + ((c >> 1) & 1), z = 2 * K + (c >> 2);
        if (x < t[3] && y < t[4] && z < t[5]) m |= (uint8_t)(1u << c);
    }
    keys[o] = gk_make(I, J, K, GT_CUBE, 0);
    vmask[o] = m;
    mol[o] = lo;
}

int gs_root_blocks_batch(const GsProblem *probs, int G, uint64_t **d_keys, uint8_t **d_vmask, int32_t **d_mol,
                         int64_t *n, cudaStream_t st)
{
    *d_keys = nullptr; *d_vmask = nullptr; *d_mol = nullptr; *n = 0;
    std::vector<int64_t> tab(6 * (size_t)G);
    int64_t total = 0;
    for (int g = 0; g < G; g++) {
        const int64_t bx = (probs[g].nroot[0] + 1) / 2, by = (probs[g].nroot[1] + 1) / 2,
                      bz = (probs[g].nroot[2] + 1) / 2;
        int64_t *t = &tab[6 * (size_t)g];
        t[0] = total; t[1] = bx; t[2] = by;
        t[3] = probs[g].nroot[0]; t[4] = probs[g].nroot[1]; t[5] = probs[g].nroot[2];
        total += bx * by * bz;
    }
    int64_t *d_tab = nullptr;
    int rc = gs_alloc((void **)&d_tab, sizeof(int64_t) * tab.size(), st);
    if (!rc) rc = gs_alloc((void **)d_keys, sizeof(uint64_t) * (size_t)total, st);
    if (!rc) rc = gs_alloc((void **)d_vmask, (size_t)total, st);
    if (!rc) rc = gs_alloc((void **)d_mol, sizeof(int32_t) * (size_t)total, st);
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(d_tab, tab.data(), sizeof(int64_t) * tab.size(), cudaMemcpyHostToDevice, st);
        if (e != cudaSuccess) rc = gs_fail_cuda(e, "root table", __FILE__, __LINE__);
    }
    if (!rc) GS_LAUNCH(k_root_blocks_batch, (unsigned)((total + 255) / 256), 256, 0, st)(d_tab, G, total, *d_keys,
                                                                                     *d_vmask, *d_mol);
    gs_free(d_tab, st);
    if (rc) {
        gs_free(*d_keys, st); gs_free(*d_vmask, st); gs_free(*d_mol, st);
        *d_keys = nullptr; *d_vmask = nullptr; *d_mol = nullptr;
        return rc;
    }
    GS_CHECK(cudaGetLastError());
    *n = total;
    return GS_OK;
}

// per-molecule decision counts: cnt[g * 5 + k] (examined, discarded,
// accepted, forced, split).  The cubes are grouped by molecule, so the lanes
// of a warp mostly share one (molecule, decision) pair and one atomic per
// pair and warp suffices.
__global__ void __launch_bounds__(256) k_level_count_mol(const uint8_t *__restrict__ dec, int64_t n,
                                                         const int32_t *__restrict__ mol,
                                                         unsigned long long *__restrict__ cnt)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const unsigned full = 0xffffffffu;
    unsigned d = q < n ? dec[q] : DEC_INVALID;
    const int g = q < n ? mol[q >> 3] : 0;
    // slot 0 (examined) for every valid cube, then the decision's own slot
    const int k = d == DEC_DISCARD ? 1 : d == DEC_ACCEPT ? 2 : d == DEC_FORCED ? 3 : d == DEC_SPLIT ? 4 : -1;
    const unsigned key0 = d != DEC_INVALID ? (unsigned)g * 8u : 0xFFFFFFFFu;
    const unsigned p0 = __match_any_sync(full, key0);
    if (key0 != 0xFFFFFFFFu && (threadIdx.x & 31) == __ffs(p0) - 1)
        atomicAdd(&cnt[(int64_t)g * 5], (unsigned long long)__popc(p0));
    const unsigned key1 = k >= 0 ? (unsigned)g * 8u + (unsigned)k : 0xFFFFFFFFu;
    const unsigned p1 = __match_any_sync(full, key1);
    if (key1 != 0xFFFFFFFFu && (threadIdx.x & 31) == __ffs(p1) - 1)
        atomicAdd(&cnt[(int64_t)g * 5 + k], (unsigned long long)__popc(p1));
}

int gs_level_count_mol(const uint8_t *d_dec, int64_t n_cubes, const int32_t *d_mol, unsigned long long *d_cnt,
                       cudaStream_t st)
{
    if (n_cubes <= 0) return GS_OK;
    GS_LAUNCH(k_level_count_mol, (unsigned)((n_cubes + 255) / 256), 256, 0, st)(d_dec, n_cubes, d_mol, d_cnt);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// accepted cubes of one compaction part to their molecules' arrays: cube j
// of the part (molecule g) goes to outs[g][j + q0 + shift[g]], q0 being the
// part's first slot among its level's accepted cubes and shift[g] the
// molecule's count over the earlier levels minus its first slot in this one
// (cap[g]: the size of molecule g's array; a slot outside it, which only
// cubes out of molecule order could give, sets GS_ST_CAPACITY instead)
__global__ void k_scatter_cubes(const uint64_t *__restrict__ acc, const int32_t *__restrict__ acc_mol, int64_t n,
                                int64_t q0, const int64_t *__restrict__ shift, uint64_t *const *__restrict__ outs,
                                const int64_t *__restrict__ cap, unsigned *status)
{
    const int64_t j = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (j >= n) return;
    const int g = acc_mol[j];
    const int64_t d = j + q0 + shift[g];
    if (d < 0 || d >= cap[g]) {
        atomicOr(status, GS_ST_CAPACITY);
        return;
    }
    outs[g][d] = acc[j];
}

int gs_scatter_cubes(const uint64_t *d_acc, const int32_t *d_acc_mol, int64_t n, int64_t q0, const int64_t *d_shift,
                     uint64_t *const *d_outs, const int64_t *d_cap, unsigned *d_status, cudaStream_t st)
{
    if (n <= 0) return GS_OK;
    GS_LAUNCH(k_scatter_cubes, (unsigned)((n + 255) / 256), 256, 0, st)(d_acc, d_acc_mol, n, q0, d_shift, d_outs,
                                                                        d_cap, d_status);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}
