// gs_cons.cu -- cubes of different sizes (section 2.3: the points of the
// neighbouring cubes that lie in the current cube are taken into its loops).
//
// With at most one level between cubes that share a face or an edge, a
// lattice vertex that lies on a face or an edge of a coarser final cube,
// without being one of its corners, takes that cube's bilinear (face) or
// linear (edge) interpolant there: the coarsest cube touching the vertex
// decides, and values are set coarse to fine, so the corners it reads are
// final.  The trilinear functions of two cubes sharing a face then agree on
// the whole face (the hanging-node constraints of conforming octree finite
// elements), so their level curves coincide and the triangulation can take
// the finer cubes' points into the coarser cube's face curve and back.
//
// A vertex whose interpolant and field value lie on different sides of c is
// a disagreement between the sizes: the coarser cubes holding it are split
// and the lattice is rebuilt (the caller loops to a fixpoint).
//
// Per vertex: lev (level of the constraining face or edge, -1 when free),
// src[4] (vertex ids: an edge's lower and upper end, or a face's corners
// (u0,w0) (u1,w0) (u0,w1) (u1,w1) in global axis order; -1 unused) and
// t[2] (fractions along the edge, or along u and w).  The interpolant
// depends only on the face or edge, not on the cube that holds it, and is
// evaluated with one rounding per operation (this file is compiled without
// FMA contraction), as in the oracle.
#include <cstring>

#include "gs_host.cuh"

__device__ __forceinline__ int64_t vert_id(const GsHash &hv, const uint64_t *slot_id, int64_t x, int64_t y, int64_t z)
{
    if (x < 0 || y < 0 || z < 0) return -1;
    const int64_t s = gs_hash_find(hv, gk_make((uint64_t)x, (uint64_t)y, (uint64_t)z, GT_VERT, 0));
    return s < 0 ? -1 : (int64_t)slot_id[s];
}

// the level-l final cubes whose closed box holds the point X (finest
// lattice); al: bit a set when X[a] lies on a level-l plane.  Each one's
// index is passed to f, which returns false to stop; returns the number
// visited.
template <typename F>
__device__ __forceinline__ int cubes_holding(const GsHash &hc, const int64_t X[3], int md, int l, int al, F f)
{
    int found = 0;
    const int sh = md - l;
    for (int c8 = 0; c8 < 8; c8++) {
        int64_t Q[3];
        bool ok = true;
        for (int a = 0; a < 3 && ok; a++) {
            const int bit = (c8 >> a) & 1, aligned = (al >> a) & 1;
            if (!aligned && bit) ok = false;
            Q[a] = (X[a] >> sh) - (aligned && bit ? 1 : 0);
            if (Q[a] < 0) ok = false;
        }
        if (!ok) continue;
        const int64_t s = gs_hash_find(hc, gk_make((uint64_t)Q[0], (uint64_t)Q[1], (uint64_t)Q[2], GT_CUBE, (unsigned)l));
        if (s >= 0) {
            found++;
            if (!f((int64_t)hc.vals[s])) break;
        }
    }
    return found;
}

__global__ void __launch_bounds__(256) k_cons_find(GsHash hc, GsHash hv, const uint64_t *__restrict__ slot_id,
                                                   const uint64_t *__restrict__ vkeys, int64_t nv, int md,
                                                   int8_t *__restrict__ lev, int32_t *__restrict__ src,
                                                   double *__restrict__ tt, int64_t *__restrict__ mark,
                                                   unsigned long long *ncons, unsigned *status)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    const uint64_t k = vkeys[i];
    const int64_t X[3] = {gk_x(k), gk_y(k), gk_z(k)};
    int L = -1;
    for (int l = 0; l < md; l++) {
        const int64_t s = (int64_t)1 << (md - l);
        int al = 0, na = 0;
        for (int a = 0; a < 3; a++)
            if ((X[a] & (s - 1)) == 0) { al |= 1 << a; na++; }
        if (na == 0) continue;
        if (!cubes_holding(hc, X, md, l, al, [](int64_t) { return false; })) continue;
        if (na == 3) break; // a corner of the coarsest cube touching it: free
        int un[2], nu = 0;
        for (int a = 0; a < 3; a++)
            if (!((al >> a) & 1)) un[nu++] = a;
        int64_t base[3];
        for (int a = 0; a < 3; a++) base[a] = ((al >> a) & 1) ? X[a] : ((X[a] >> (md - l)) << (md - l));
        L = l;
        for (int q = 0; q < 2; q++)
            tt[2 * i + q] = q < nu ? __ddiv_rn((double)(X[un[q]] - base[un[q]]), (double)s) : 0.0;
        const int nsrc = nu == 1 ? 2 : 4;
        for (int q = 0; q < 4; q++) {
            int32_t id = -1;
            if (q < nsrc) {
                int64_t Y[3] = {base[0], base[1], base[2]};
                for (int b = 0; b < nu; b++) Y[un[b]] += ((q >> b) & 1) ? s : 0;
                const int64_t v = vert_id(hv, slot_id, Y[0], Y[1], Y[2]);
                if (v < 0) atomicOr(status, GS_ST_LOOKUP);
                id = (int32_t)v;
                if (mark && v >= 0) mark[v] = 1;
            }
            src[4 * i + q] = id;
        }
        if (mark) mark[i] = 1;
        atomicAdd(ncons, 1ull);
        break;
    }
    lev[i] = (int8_t)L;
}

// values of the vertices constrained at level l from their sources (final
// already).  err (nullable): FP32 bounds, the interpolant's bound is the same
// interpolant of its sources' bounds (a convex combination; the FP64
// rounding of the interpolation is far below them), exact sources give 0.
// mark (nullable): where |value - c| is within 4 bounds, the sources are
// marked for FP64.  split (nullable): count a sign disagreement with the
// vertex's own field value and mark the level-l cubes holding the vertex
// (cnt = 8).
// (over the level-l group of the constrained-vertex list: ids[0 .. n))
__global__ void __launch_bounds__(256) k_cons_apply(int l, int md, double c, GsHash hc,
                                                    const uint64_t *__restrict__ vkeys, const int32_t *__restrict__ ids,
                                                    int64_t n, const int32_t *__restrict__ src,
                                                    const double *__restrict__ tt, double *__restrict__ phi,
                                                    float *__restrict__ err, int64_t *__restrict__ mark,
                                                    int64_t *__restrict__ split, unsigned long long *nflip)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int64_t i = ids[q];
    const int32_t *S = src + 4 * i;
    const double t0 = tt[2 * i], t1 = tt[2 * i + 1];
    double psi;
    float e = 0.f;
    if (S[2] < 0) {
        const double a = phi[S[0]], b = phi[S[1]];
        psi = __dadd_rn(a, __dmul_rn(t0, __dsub_rn(b, a)));
        if (err) e = (float)((1.0 - t0) * err[S[0]] + t0 * err[S[1]]);
    } else {
        const double q00 = phi[S[0]], q10 = phi[S[1]], q01 = phi[S[2]], q11 = phi[S[3]];
        const double e0 = __dadd_rn(q00, __dmul_rn(t0, __dsub_rn(q10, q00)));
        const double e1 = __dadd_rn(q01, __dmul_rn(t0, __dsub_rn(q11, q01)));
        psi = __dadd_rn(e0, __dmul_rn(t1, __dsub_rn(e1, e0)));
        if (err)
            e = (float)((1.0 - t0) * (1.0 - t1) * err[S[0]] + t0 * (1.0 - t1) * err[S[1]] +
                        (1.0 - t0) * t1 * err[S[2]] + t0 * t1 * err[S[3]]);
    }
    if (err && e > 0.f) e = e * 1.0001f + 1e-12f;  // the bound's own rounding
    if (mark && fabs(psi - c) <= 4.0 * (double)e)
        for (int q = 0; q < 4; q++)
            if (S[q] >= 0) mark[S[q]] = 1;
    if (split && ((psi >= c) != (phi[i] >= c))) {
        atomicAdd(nflip, 1ull);
        const uint64_t k = vkeys[i];
        const int64_t X[3] = {gk_x(k), gk_y(k), gk_z(k)};
        const int64_t s = (int64_t)1 << (md - l);
        int al = 0;
        for (int a = 0; a < 3; a++)
            if ((X[a] & (s - 1)) == 0) al |= 1 << a;
        cubes_holding(hc, X, md, l, al, [&](int64_t ci) { split[ci] = 8; return true; });
    }
    phi[i] = psi;
    if (err) err[i] = e;
}

// marks on vertices constrained at level l pass to their sources (run from
// the finest constraint level to the coarsest)
__global__ void __launch_bounds__(256) k_cons_mark_up(const int32_t *__restrict__ ids, int64_t n,
                                                      const int32_t *__restrict__ src, int64_t *__restrict__ mark)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int64_t i = ids[q];
    if (!mark[i]) return;
    for (int q = 0; q < 4; q++)
        if (src[4 * i + q] >= 0) mark[src[4 * i + q]] = 1;
}

// a cube with a mixed-size contact: a constrained corner (a coarser cube
// touches it) or a lattice vertex at an edge midpoint or face centre (a
// finer one does)
__global__ void __launch_bounds__(256) k_mixed_flags(const uint64_t *__restrict__ cubes, int64_t n,
                                                     const int32_t *__restrict__ cvid, const int8_t *__restrict__ lev,
                                                     GsHash hv, const uint64_t *__restrict__ slot_id, int md,
                                                     uint8_t *__restrict__ mixed, unsigned long long *nmixed)
{
    const int64_t ci = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= n) return;
    int f = 0;
    for (int v = 0; v < 8 && !f; v++) f = lev[cvid[8 * ci + v]] >= 0;
    const uint64_t k = cubes[ci];
    const int l = (int)gk_level(k);
    if (!f && l < md) {
        const int64_t s = (int64_t)1 << (md - l), h = s >> 1;
        const int64_t C[3] = {gk_x(k) * s, gk_y(k) * s, gk_z(k) * s};
        // the 18 points at (0|h|s) offsets with exactly one or two h's
        for (int d = 0; d < 27 && !f; d++) {
            const int o[3] = {d % 3, (d / 3) % 3, d / 9};
            const int nh = (o[0] == 1) + (o[1] == 1) + (o[2] == 1);
            if (nh == 0 || nh == 3) continue;
            int64_t P[3];
            for (int a = 0; a < 3; a++) P[a] = C[a] + (o[a] == 0 ? 0 : (o[a] == 1 ? h : s));
            f = vert_id(hv, slot_id, P[0], P[1], P[2]) >= 0;
        }
    }
    mixed[ci] = (uint8_t)f;
    if (f) atomicAdd(nmixed, 1ull);
}

// constrained vertices keep their interpolants: no FP64 re-evaluation of
// the field there (it would overwrite them)
__global__ void k_cons_unmark(const int32_t *__restrict__ ids, int64_t n, int64_t *__restrict__ mark)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q < n) mark[ids[q]] = 0;
}

// adjoint of the level-l constraints: each passes its adjoint on to its
// sources with the interpolation weights (fine to coarse)
__global__ void __launch_bounds__(256) k_cons_adjoint(const int32_t *__restrict__ ids, int64_t n,
                                                      const int32_t *__restrict__ src, const double *__restrict__ tt,
                                                      double *__restrict__ lam)
{
    const int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    const int64_t i = ids[q];
    const double g = lam[i];
    lam[i] = 0.0;
    if (g == 0.0) return;
    const int32_t *S = src + 4 * i;
    const double tu = tt[2 * i], tw = tt[2 * i + 1];
    if (S[2] < 0) {
        atomicAdd(&lam[S[0]], g * (1.0 - tu));
        atomicAdd(&lam[S[1]], g * tu);
    } else {
        atomicAdd(&lam[S[0]], g * (1.0 - tu) * (1.0 - tw));
        atomicAdd(&lam[S[1]], g * tu * (1.0 - tw));
        atomicAdd(&lam[S[2]], g * (1.0 - tu) * tw);
        atomicAdd(&lam[S[3]], g * tu * tw);
    }
}

__global__ void k_fill_i64(int64_t *__restrict__ a, int64_t n, int64_t v)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) a[i] = v;
}

// ---------------------------------------------------------------- host
int gs_fill_i64(int64_t *d_a, int64_t n, int64_t v, cudaStream_t st)
{
    if (n <= 0) return GS_OK;
    GS_LAUNCH(k_fill_i64, (unsigned)((n + 255) / 256), 256, 0, st)(d_a, n, v);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

int gs_cons_alloc(GsCons *K, int64_t nv, cudaStream_t st)
{
    K->lev = nullptr; K->src = nullptr; K->t = nullptr; K->nv = nv; K->ncons = 0; K->list = nullptr;
    memset(K->loff, 0, sizeof(K->loff));
    int rc = gs_alloc((void **)&K->lev, (size_t)(nv + 1), st);
    if (!rc) rc = gs_alloc((void **)&K->src, sizeof(int32_t) * 4 * (size_t)(nv + 1), st);
    if (!rc) rc = gs_alloc((void **)&K->t, sizeof(double) * 2 * (size_t)(nv + 1), st);
    if (rc) gs_cons_free(K, st);
    return rc;
}

void gs_cons_free(GsCons *K, cudaStream_t st)
{
    gs_free(K->lev, st); gs_free(K->src, st); gs_free(K->t, st); gs_free(K->list, st);
    K->lev = nullptr; K->src = nullptr; K->t = nullptr; K->list = nullptr;
}

__global__ void k_cons_flag(const int8_t *__restrict__ lev, int64_t nv, int l, int64_t *__restrict__ flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv) flag[i] = lev[i] == l;
}
__global__ void k_cons_group(const int64_t *__restrict__ off, int64_t nv, int32_t *__restrict__ out)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < nv && off[i + 1] != off[i]) out[off[i]] = (int32_t)i;
}

// the constrained vertices grouped by level, each group in vertex order
// (a flag, scan and scatter per level)
static int cons_list(GsCons *K, int md, cudaStream_t st)
{
    memset(K->loff, 0, sizeof(K->loff));
    gs_free(K->list, st);
    K->list = nullptr;
    if (K->ncons <= 0) return GS_OK;
    int64_t *flag = nullptr, *tot = nullptr;
    int rc = gs_alloc((void **)&K->list, sizeof(int32_t) * (size_t)K->ncons, st);
    if (!rc) rc = gs_alloc((void **)&flag, sizeof(int64_t) * (size_t)(K->nv + 1), st);
    if (!rc) rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
    const unsigned nb = (unsigned)((K->nv + 255) / 256);
    int64_t base = 0;
    for (int l = 0; l < md && l < 21 && !rc; l++) {
        K->loff[l] = base;
        cudaMemsetAsync(flag + K->nv, 0, sizeof(int64_t), st);
        GS_LAUNCH(k_cons_flag, nb, 256, 0, st)(K->lev, K->nv, l, flag);
        rc = gs_scan_i64(flag, K->nv + 1, tot, st);
        int64_t cnt = 0;
        if (!rc) {
            cudaError_t e = cudaMemcpyAsync(&cnt, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = gs_sync(st);
            if (e != cudaSuccess) rc = gs_fail_cuda(e, "constraint groups", __FILE__, __LINE__);
        }
        if (!rc && base + cnt > K->ncons) rc = gs_fail(GS_ERR_DEVICE_STATUS, "constraint groups exceed their count");
        if (!rc && cnt > 0) GS_LAUNCH(k_cons_group, nb, 256, 0, st)(flag, K->nv, K->list + base);
        base += cnt;
    }
    for (int l = md < 21 ? md : 21; l < 22; l++) K->loff[l] = base;
    gs_free(flag, st);
    gs_free(tot, st);
    if (!rc && base != K->ncons) rc = gs_fail(GS_ERR_DEVICE_STATUS, "constraint groups: %lld of %lld vertices",
                                              (long long)base, (long long)K->ncons);
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

int gs_cons_find(GsCons *K, const GsHash &hc, const GsHash &hv, const uint64_t *d_slot_id, const uint64_t *d_vkeys,
                 int md, int64_t *d_mark, unsigned long long *d_scratch, unsigned *d_status, cudaStream_t st)
{
    K->ncons = 0;
    if (K->nv <= 0) return GS_OK;
    GS_CHECK(cudaMemsetAsync(d_scratch, 0, sizeof(unsigned long long), st));
    GS_LAUNCH(k_cons_find, (unsigned)((K->nv + 255) / 256), 256, 0, st)(hc, hv, d_slot_id, d_vkeys, K->nv, md, K->lev,
                                                                        K->src, K->t, d_mark, d_scratch, d_status);
    unsigned long long h = 0;
    GS_CHECK(cudaMemcpyAsync(&h, d_scratch, sizeof(h), cudaMemcpyDeviceToHost, st));
    GS_CHECK(gs_sync(st));
    K->ncons = (int64_t)h;
    return cons_list(K, md, st);
}

int gs_cons_apply(const GsCons &K, const GsHash &hc, const uint64_t *d_vkeys, int md, double c, double *d_phi,
                  float *d_err, int64_t *d_mark, int64_t *d_split, int64_t *n_flip, unsigned long long *d_scratch,
                  cudaStream_t st)
{
    if (n_flip) *n_flip = 0;
    if (K.nv <= 0 || K.ncons == 0) return GS_OK;
    if (d_split) GS_CHECK(cudaMemsetAsync(d_scratch, 0, sizeof(unsigned long long), st));
    for (int l = 0; l < md && l < 21; l++) {
        const int64_t n = K.loff[l + 1] - K.loff[l];
        if (n > 0)
            GS_LAUNCH(k_cons_apply, (unsigned)((n + 255) / 256), 256, 0, st)(l, md, c, hc, d_vkeys, K.list + K.loff[l],
                                                                            n, K.src, K.t, d_phi, d_err, d_mark,
                                                                            d_split, d_scratch);
    }
    if (d_split && n_flip) {
        unsigned long long h = 0;
        GS_CHECK(cudaMemcpyAsync(&h, d_scratch, sizeof(h), cudaMemcpyDeviceToHost, st));
        GS_CHECK(gs_sync(st));
        *n_flip = (int64_t)h;
    }
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

int gs_mixed_flags(const GsCons &K, const uint64_t *d_cubes, int64_t n, const int32_t *d_cvid, const GsHash &hv,
                   const uint64_t *d_slot_id, int md, uint8_t *d_mixed, int64_t *n_mixed,
                   unsigned long long *d_scratch, cudaStream_t st)
{
    *n_mixed = 0;
    if (n <= 0) return GS_OK;
    GS_CHECK(cudaMemsetAsync(d_scratch, 0, sizeof(unsigned long long), st));
    GS_LAUNCH(k_mixed_flags, (unsigned)((n + 255) / 256), 256, 0, st)(d_cubes, n, d_cvid, K.lev, hv, d_slot_id, md,
                                                                       d_mixed, d_scratch);
    unsigned long long h = 0;
    GS_CHECK(cudaMemcpyAsync(&h, d_scratch, sizeof(h), cudaMemcpyDeviceToHost, st));
    GS_CHECK(gs_sync(st));
    *n_mixed = (int64_t)h;
    return GS_OK;
}

int gs_cons_mark_up(const GsCons &K, int md, int64_t *d_mark, cudaStream_t st)
{
    if (K.nv <= 0 || K.ncons == 0) return GS_OK;
    for (int l = (md < 21 ? md : 21) - 1; l >= 0; l--) {
        const int64_t n = K.loff[l + 1] - K.loff[l];
        if (n > 0)
            GS_LAUNCH(k_cons_mark_up, (unsigned)((n + 255) / 256), 256, 0, st)(K.list + K.loff[l], n, K.src, d_mark);
    }
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}


int gs_cons_unmark(const GsCons &K, int64_t *d_mark, cudaStream_t st)
{
    if (K.nv <= 0 || K.ncons == 0) return GS_OK;
    GS_LAUNCH(k_cons_unmark, (unsigned)((K.ncons + 255) / 256), 256, 0, st)(K.list, K.ncons, d_mark);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

int gs_cons_adjoint(const GsCons &K, int md, double *d_lambda, cudaStream_t st)
{
    if (K.nv <= 0 || K.ncons == 0) return GS_OK;
    for (int l = (md < 21 ? md : 21) - 1; l >= 0; l--) {
        const int64_t n = K.loff[l + 1] - K.loff[l];
        if (n > 0)
            GS_LAUNCH(k_cons_adjoint, (unsigned)((n + 255) / 256), 256, 0, st)(K.list + K.loff[l], n, K.src, K.t,
                                                                              d_lambda);
    }
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}
