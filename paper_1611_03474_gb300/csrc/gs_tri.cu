// gs_tri.cu -- per-cube trilinear surface and its triangulation (section 2.3).
//
// For each accepted cube whose corner values straddle c, the trilinear
// interpolant g of eq linear1 is cut by g = c:
//   * edge points solve g = c on the 12 edges (eq intersection);
//   * fold lines {g = c, dg/ds = 0} (eq fold1) are segments parallel to an
//     axis s; their ends on the two faces normal to s are the extreme points
//     (eq curve); fold lines of two axes meet at critical points (eq
//     critical), which for a trilinear g occur whenever both lie in one slice;
//   * on each face the bilinear level curve joins edge points along
//     hyperbola branches (asymptotic decider) and takes, in order, the
//     extreme points of this cube and of the same-size neighbour across the
//     face ("points of the neighbouring cubes are considered");
//   * the loops so formed, cut along all fold segments, bound single-valued
//     pieces, each triangulated by ear clipping in the coordinate plane of
//     its largest projected area (two-ears theorem).
// Decisions that two cubes sharing a face must agree on (edge points, fold
// roots, face arcs) are taken by the same non-inlined functions on the same
// values in the face's global axis order.
//
// Thread per cube, two passes over the same code: count (triangles,
// points) and emit into scan-allocated buffers.  Bounded loops only; an
// inconsistency sets a counter and skips the cube.  This file is compiled
// without FMA contraction (-fmad=false): geometric predicates (orientation,
// in-square and branch tests) then round each product and sum once, so
// exactly degenerate configurations are recognised as such.
#include "gs_host.cuh"

#define TP_MAX 48      // points of a cube whose neighbours across faces and edges have its size
#define TP_MIX 64      // points of a cube with neighbours of another size
#define FP_MIX 20      // points inserted into one face curve (another size)
#define POLY_MAX 96

struct TPt {
    double p[3];      // cube-local coordinates in [0,1]
    uint64_t key;
    signed char kind; // 0 edge, 1 own extreme, 2 neighbour extreme, 3 critical
    signed char nb[4];
    signed char fa, fb, rh;
};

__device__ __forceinline__ void axes_other(int a, int &u, int &v)
{
    u = (a == 0) ? 1 : 0;
    v = (a == 2) ? 1 : 2;
}

__device__ __forceinline__ double corner(const double *g, int bx, int by, int bz) { return g[bx + 2 * by + 4 * bz]; }

// roots (u,v) in the open unit square of {B = 0, A = c} for g = A + s B along axis a
// roots (u, v) of the fold line of axis a in (0,1)^2 (in (-slack, 1+slack)^2
// when slack > 0, for the error marks)
// sgn: bit v = (g[v] >= c), or -1 to compare here
__device__ __noinline__ int fold_solve(const double *g, int a, double c, double *ru, double *rv, double slack = 0.0,
                                       int sgn = -1)
{
    int ua, va;
    axes_other(a, ua, va);
    if (sgn < 0) {
        sgn = 0;
        for (int v = 0; v < 8; v++) sgn |= (g[v] >= c ? 1 : 0) << v;
    }
    int nlo = 0, nup = 0;
    for (int k = 0; k < 4; k++) {
        int b[3];
        b[a] = 0; b[ua] = k & 1; b[va] = k >> 1;
        nlo += (sgn >> (b[0] + 2 * b[1] + 4 * b[2])) & 1;
        b[a] = 1;
        nup += (sgn >> (b[0] + 2 * b[1] + 4 * b[2])) & 1;
    }
    if (nlo == 0 || nlo == 4 || nup == 0 || nup == 4) return 0;
    double lo[4], up[4];  // face s=0 and s=1 values at (u,v) = (0,0),(1,0),(0,1),(1,1)
    for (int k = 0; k < 4; k++) {
        int b[3];
        b[a] = 0; b[ua] = k & 1; b[va] = k >> 1;
        lo[k] = corner(g, b[0], b[1], b[2]);
        b[a] = 1;
        up[k] = corner(g, b[0], b[1], b[2]);
    }
    // A - c = p0 + p1 u + p2 v + p3 uv ; B = q0 + q1 u + q2 v + q3 uv
    // monomial coefficients, summed left to right (the face's corner order)
    double p0 = lo[0] - c, p1 = lo[1] - lo[0], p2 = lo[2] - lo[0], p3 = lo[3] - lo[1] - lo[2] + lo[0];
    double d0 = up[0] - lo[0], d1 = up[1] - lo[1], d2 = up[2] - lo[2], d3 = up[3] - lo[3];
    double q0 = d0, q1 = d1 - d0, q2 = d2 - d0, q3 = d3 - d1 - d2 + d0;
    if (q0 == 0.0 && q1 == 0.0 && q2 == 0.0 && q3 == 0.0) return 0;
    // eliminate v: (p0 + p1 u)(q2 + q3 u) - (p2 + p3 u)(q0 + q1 u) = 0
    double A2 = p1 * q3 - p3 * q1;
    double A1 = p0 * q3 + p1 * q2 - p2 * q1 - p3 * q0;
    double A0 = p0 * q2 - p2 * q0;
    double us[2];
    int nu = 0;
    if (A2 == 0.0) {
        if (A1 != 0.0) us[nu++] = -A0 / A1;
    } else {
        double disc = A1 * A1 - 4.0 * A2 * A0;
        if (disc >= 0.0) {
            double sq = sqrt(disc);
            double w = A1 >= 0.0 ? -0.5 * (A1 + sq) : -0.5 * (A1 - sq);
            if (w != 0.0) {
                us[nu++] = w / A2;
                double u2 = A0 / w;
                if (u2 != us[0]) us[nu++] = u2;
            } else {
                us[nu++] = 0.0;
            }
        }
    }
    double sp = fabs(p0) + fabs(p1) + fabs(p2) + fabs(p3), sq_ = fabs(q0) + fabs(q1) + fabs(q2) + fabs(q3);
    int nr = 0;
    for (int i = 0; i < nu; i++) {
        double u = us[i];
        if (!(u > -slack && u < 1.0 + slack)) continue;
        double denB = q2 + q3 * u, denA = p2 + p3 * u;
        double cand0, cand1;
        bool h0, h1;
        if (fabs(denB) >= fabs(denA)) {
            h0 = denB != 0.0; cand0 = h0 ? -(q0 + q1 * u) / denB : 0.0;
            h1 = denA != 0.0; cand1 = h1 ? -(p0 + p1 * u) / denA : 0.0;
        } else {
            h0 = denA != 0.0; cand0 = h0 ? -(p0 + p1 * u) / denA : 0.0;
            h1 = denB != 0.0; cand1 = h1 ? -(q0 + q1 * u) / denB : 0.0;
        }
        for (int t = 0; t < 2; t++) {
            bool has = t ? h1 : h0;
            double v = t ? cand1 : cand0;
            if (!has || !(v > -slack && v < 1.0 + slack)) continue;
            if (fabs(p0 + p1 * u + p2 * v + p3 * u * v) > 1e-9 * sp) continue;
            if (fabs(q0 + q1 * u + q2 * v + q3 * u * v) > 1e-9 * sq_) continue;
            ru[nr] = u; rv[nr] = v; nr++;
            break;
        }
    }
    if (nr == 2 && (ru[1] < ru[0] || (ru[1] == ru[0] && rv[1] < rv[0]))) {
        double t = ru[0]; ru[0] = ru[1]; ru[1] = t;
        t = rv[0]; rv[0] = rv[1]; rv[1] = t;
    }
    return nr;
}

// face decision in the face's (u,v) frame from h[u + 2v]: returns the number
// of arcs (0,1,2); for two arcs sets around00 (arcs cut off corners 00 and
// 11) and the saddle's u coordinate
// fs: bit k = (h[k] >= c), or -1 to compare here
__device__ __noinline__ int face_arcs(const double *h, double c, int &around00, double &us, int fs = -1)
{
    if (fs < 0) fs = (h[0] >= c ? 1 : 0) | (h[1] >= c ? 2 : 0) | (h[2] >= c ? 4 : 0) | (h[3] >= c ? 8 : 0);
    int nin = __popc(fs);
    around00 = 0;
    us = 0.0;
    if (nin == 0 || nin == 4) return 0;
    // diagonal pattern: corners 0 and 3 on one side, 1 and 2 on the other
    if (fs != 9 && fs != 6) return 1;
    double den = h[0] - h[1] - h[2] + h[3];
    double hs = (h[0] * h[3] - h[1] * h[2]) / den;
    us = (h[0] - h[2]) / den;
    bool in00 = fs & 1;
    bool sep = hs < c;
    around00 = (in00 == sep) ? 1 : 0;
    return 2;
}

// Where a cube's output goes: triangles are written while fewer than
// tri_cap have been produced, points only if all of them fit in pt_cap.  The
// final pass writes at the scanned offsets with unbounded caps; the first
// pass writes into a fixed per-cube staging slot (caps TRI_STAGE_T,
// TRI_STAGE_P), so only cubes that overflow it are traced a second time.
struct TriOut {
    uint64_t *tri_keys;   // [3] per triangle
    uint64_t *pt_keys;
    double *pt_xyz;
    int64_t tri_off, pt_off;
    int tri_cap, pt_cap;
    int ntri, npt;
};
#define TRI_STAGE_T 4
#define TRI_STAGE_P 6

__device__ __forceinline__ void put_tri(TriOut &o, uint64_t a, uint64_t b, uint64_t c)
{
    if (o.ntri < o.tri_cap) {
        uint64_t *d = o.tri_keys + 3 * (o.tri_off + o.ntri);
        d[0] = a; d[1] = b; d[2] = c;
    }
    o.ntri++;
}

__device__ __forceinline__ double orient(const double *a, const double *b, const double *c, int i, int j)
{
    return (b[i] - a[i]) * (c[j] - a[j]) - (b[j] - a[j]) * (c[i] - a[i]);
}

// ear clipping of one piece (indices into pts), CCW seen from outside; pf
// holds the points' coordinates rounded to FP32
__device__ void clip_piece(const TPt *pts, const float (*pf)[3], const unsigned char *poly, int n, TriOut &o,
                           unsigned long long *degen)
{
    // Newell normal; the piece is projected along its largest component.
    // FP32 first: with coordinates in [0,1] each term is at most 2 and carries
    // at most 7.2e-7 of rounding, the partial sums at most 2n * 6e-8 each, so
    // every component lies within errM of its exact value.  When the largest
    // leads the others by more than 2 errM, the axis and the sign are those of
    // the exact (and the FP64) normal; otherwise FP64 decides.
    float M0 = 0.f, M1 = 0.f, M2 = 0.f;
    for (int i = 0; i < n; i++) {
        const float *p = pf[poly[i]], *q = pf[poly[i + 1 == n ? 0 : i + 1]];
        M0 += (p[1] - q[1]) * (p[2] + q[2]);
        M1 += (p[2] - q[2]) * (p[0] + q[0]);
        M2 += (p[0] - q[0]) * (p[1] + q[1]);
    }
    const float errM = (float)n * (1e-6f + 1.5e-7f * (float)n);
    const float b0 = fabsf(M0), b1 = fabsf(M1), b2 = fabsf(M2);
    int k;
    double sg;
    const int kf = b0 >= b1 ? (b0 >= b2 ? 0 : 2) : (b1 >= b2 ? 1 : 2);
    const float top = kf == 0 ? b0 : (kf == 1 ? b1 : b2);
    const float second = kf == 0 ? fmaxf(b1, b2) : (kf == 1 ? fmaxf(b0, b2) : fmaxf(b0, b1));
    if (top - second > 2.f * errM && top > errM) {
        k = kf;
        sg = (kf == 0 ? M0 : (kf == 1 ? M1 : M2)) >= 0.f ? 1.0 : -1.0;
    } else {
        double N0 = 0, N1 = 0, N2 = 0;
        for (int i = 0; i < n; i++) {
            const double *p = pts[poly[i]].p, *q = pts[poly[i + 1 == n ? 0 : i + 1]].p;
            N0 += (p[1] - q[1]) * (p[2] + q[2]);
            N1 += (p[2] - q[2]) * (p[0] + q[0]);
            N2 += (p[0] - q[0]) * (p[1] + q[1]);
        }
        k = 0;
        double best = fabs(N0);
        if (fabs(N1) > best) { k = 1; best = fabs(N1); }
        if (fabs(N2) > best) k = 2;
        double Nk = k == 0 ? N0 : (k == 1 ? N1 : N2);
        sg = Nk >= 0 ? 1.0 : -1.0;
    }
    int ia = (k + 1) % 3, ib = (k + 2) % 3;
    unsigned char v[POLY_MAX];
    for (int i = 0; i < n; i++) v[i] = poly[i];
    // Orientation signs, filtered in FP32: the points' local coordinates lie
    // in [0,1], so rounding them to float moves each difference by at most
    // 1.8e-7 and each product by 1.8e-7 times the other factor; when the
    // FP32 value exceeds that bound (with margin) its sign is the exact sign
    // and the FP64 predicate's.  Otherwise the FP64 predicate decides.
    float qa[TP_MIX], qb[TP_MIX];
    for (int i = 0; i < n; i++) {
        qa[poly[i]] = pf[poly[i]][ia];
        qb[poly[i]] = pf[poly[i]][ib];
    }
    auto osign = [&](int a, int b, int c) -> int {
        float d1 = qa[b] - qa[a], d2 = qb[c] - qb[a], d3 = qb[b] - qb[a], d4 = qa[c] - qa[a];
        float p1 = d1 * d2, p2 = d3 * d4, vv = p1 - p2;
        float err = 4e-7f * (fabsf(d1) + fabsf(d2) + fabsf(d3) + fabsf(d4)) + 3e-7f * (fabsf(p1) + fabsf(p2)) + 1e-13f;
        int s32 = vv > err ? 1 : (vv < -err ? -1 : 0);
        if (s32 != 0) return sg > 0 ? s32 : -s32;
        double o = sg * orient(pts[a].p, pts[b].p, pts[c].p, ia, ib);
        return o > 0 ? 1 : (o < 0 ? -1 : 0);
    };
    int m = n;
    int guard = 0;
    while (m > 3 && guard++ < POLY_MAX) {
        int pick = -1, fall = -1;
        for (int i = 0; i < m; i++) {
            int a = v[i == 0 ? m - 1 : i - 1], b = v[i], c = v[i + 1 == m ? 0 : i + 1];
            if (fall < 0 || pts[b].key < pts[v[fall]].key) fall = i;
            if (!(osign(a, b, c) > 0)) continue;
            bool empty = true;
            for (int jx = 0; jx < m && empty; jx++) {
                int d = v[jx];
                if (d == a || d == b || d == c) continue;
                if (osign(a, b, d) >= 0 && osign(b, c, d) >= 0 && osign(c, a, d) >= 0) empty = false;
            }
            if (!empty) continue;
            if (pick < 0 || pts[b].key < pts[v[pick]].key) pick = i;
        }
        if (pick < 0) { pick = fall; if (degen) atomicAdd(degen, 1ull); }
        int a = v[pick == 0 ? m - 1 : pick - 1], b = v[pick], c = v[pick + 1 == m ? 0 : pick + 1];
        if (a != b && b != c && a != c) put_tri(o, pts[a].key, pts[b].key, pts[c].key);
        for (int t = pick; t < m - 1; t++) v[t] = v[t + 1];
        m--;
    }
    if (m == 3 && v[0] != v[1] && v[1] != v[2] && v[0] != v[2]) put_tri(o, pts[v[0]].key, pts[v[1]].key, pts[v[2]].key);
}

template <int CAP>
__device__ __forceinline__ int64_t add_pt(TPt *pts, int &np, int kind)
{
    if (np >= CAP) return -1;
    TPt &p = pts[np];
    p.kind = (signed char)kind;
    p.nb[0] = p.nb[1] = p.nb[2] = p.nb[3] = -1;
    p.fa = p.fb = p.rh = 0;
    return np++;
}

// world coordinate at fraction f of the level-lvl edge starting at lattice
// index i on axis a (the index's lattice coordinate when f is 0 or 1)
__device__ __forceinline__ double wfrac(const TriCtx &X, int a, int64_t i, int lvl, double f)
{
    const int64_t s = (int64_t)1 << (X.max_depth - lvl);
    const double lo = __dadd_rn(X.origin[a], __dmul_rn((double)(i * s), X.min_edge));
    if (f == 0.0) return lo;
    if (f == 1.0) return __dadd_rn(X.origin[a], __dmul_rn((double)((i + 1) * s), X.min_edge));
    return __dadd_rn(lo, __dmul_rn(f, ldexp(X.min_edge, X.max_depth - lvl)));
}
// world coordinate of finest-lattice index L on axis a
__device__ __forceinline__ double wlat(const TriCtx &X, int a, int64_t L)
{
    return __dadd_rn(X.origin[a], __dmul_rn((double)L, X.min_edge));
}
__device__ __forceinline__ int64_t tri_vert(const TriCtx &X, int64_t x, int64_t y, int64_t z)
{
    if (x < 0 || y < 0 || z < 0) return -1;
    const int64_t s = gs_hash_find(X.hv, gk_make((uint64_t)x, (uint64_t)y, (uint64_t)z, GT_VERT, 0));
    return s < 0 ? -1 : (int64_t)X.vslot_id[s];
}
__device__ __forceinline__ int64_t tri_cube_at(const TriCtx &X, int64_t x, int64_t y, int64_t z, int lvl)
{
    if (x < 0 || y < 0 || z < 0) return -1;
    const int64_t s = gs_hash_find(X.hc, gk_make((uint64_t)x, (uint64_t)y, (uint64_t)z, GT_CUBE, (unsigned)lvl));
    return s < 0 ? -1 : (int64_t)X.hc.vals[s];
}
// fold roots of axis a of cube q (from the table when there is one)
__device__ __forceinline__ int cube_fold_roots(const TriCtx &X, int64_t q, int a, double *ru, double *rv)
{
    if (X.fcount) {
        const int nn = X.fcount[q * 4 + a];
        for (int r = 0; r < nn; r++) {
            ru[r] = X.froot[q * 12 + 4 * a + 2 * r];
            rv[r] = X.froot[q * 12 + 4 * a + 2 * r + 1];
        }
        return nn;
    }
    double gq[8];
    for (int v = 0; v < 8; v++) gq[v] = X.phi[X.cvid[q * 8 + v]];
    return fold_solve(gq, a, X.c, ru, rv);
}

// Points across face (a, sd) of cube C (level lvl) that has no neighbour of
// its own size there: the finer neighbours' fold ends and inner half-line
// points, or the coarser neighbour's fold ends inside this face.  All of
// them lie on this face's level curve (constrained vertex values make the
// finer faces' and this face's values one bilinear function).  Returns 1 on
// an inconsistency.
__device__ __noinline__ int tri_mixed_face(const TriCtx &X, const int64_t *C, int lvl, int a, int sd, bool fine_ok,
                                           TPt *pts, double (*pw)[3], int &np, signed char *fp, int &nfp)
{
    int ua, va;
    axes_other(a, ua, va);
    const double c = X.c;
    const int64_t sc = (int64_t)1 << (X.max_depth - lvl), s2 = sc >> 1;
    int64_t N[3] = {C[0], C[1], C[2]};
    N[a] += sd ? 1 : -1;
    if (N[a] < 0) return 0;
    const int side_n = sd ? 0 : 1;          // the neighbour's side of the shared plane
    const int64_t plane = (C[a] + sd) * sc; // finest-lattice coordinate of the face
    if (fine_ok) {
        int64_t tq[4], T[4][3];
        int ntile = 0;
        for (int iv = 0; iv < 2; iv++)
            for (int iu = 0; iu < 2; iu++) {
                const int q = iu + 2 * iv;
                T[q][a] = 2 * N[a] + side_n; T[q][ua] = 2 * C[ua] + iu; T[q][va] = 2 * C[va] + iv;
                tq[q] = tri_cube_at(X, T[q][0], T[q][1], T[q][2], lvl + 1);
                ntile += tq[q] >= 0;
            }
        if (ntile > 0) {
            for (int iv = 0; iv < 2; iv++)
                for (int iu = 0; iu < 2; iu++) {
                    const int q = iu + 2 * iv;
                    if (tq[q] < 0) continue;
                    double tu[2], tv[2];
                    const int nn = cube_fold_roots(X, tq[q], a, tu, tv);
                    for (int r = 0; r < nn; r++) {
                        const int id = (int)add_pt<TP_MIX>(pts, np, 2);
                        if (id < 0 || nfp >= FP_MIX) return 1;
                        pts[id].p[a] = sd;
                        pts[id].p[ua] = __dmul_rn(__dadd_rn((double)iu, tu[r]), 0.5);
                        pts[id].p[va] = __dmul_rn(__dadd_rn((double)iv, tv[r]), 0.5);
                        int64_t L[3] = {T[q][0] * s2, T[q][1] * s2, T[q][2] * s2};
                        L[a] = plane;
                        pts[id].key = gk_make(L[0], L[1], L[2], 8u + 4u * a + 2u * (side_n == 0 ? 1u : 0u) + (unsigned)r,
                                              (unsigned)(lvl + 1));
                        pw[id][a] = wlat(X, a, plane);
                        pw[id][ua] = wfrac(X, ua, T[q][ua], lvl + 1, tu[r]);
                        pw[id][va] = wfrac(X, va, T[q][va], lvl + 1, tv[r]);
                        fp[nfp++] = (signed char)id;
                    }
                }
            // inner half-lines: along u at v = 1/2 (halves k), then along v at
            // u = 1/2; each is an edge of the tiles on either side of it
            for (int dir = 0; dir < 2; dir++)
                for (int k = 0; k < 2; k++) {
                    const int along = dir ? va : ua, across = dir ? ua : va;
                    const bool has = dir ? (tq[2 * k] >= 0 || tq[1 + 2 * k] >= 0) : (tq[k] >= 0 || tq[k + 2] >= 0);
                    if (!has) continue;
                    int64_t L0[3];
                    L0[a] = plane;
                    L0[along] = C[along] * sc + k * s2;
                    L0[across] = C[across] * sc + s2;
                    int64_t L1[3] = {L0[0], L0[1], L0[2]};
                    L1[along] += s2;
                    const int64_t ia = tri_vert(X, L0[0], L0[1], L0[2]), ib = tri_vert(X, L1[0], L1[1], L1[2]);
                    if (ia < 0 || ib < 0) return 1;
                    const double ga = X.phi[ia], gb = X.phi[ib];
                    if ((ga >= c) == (gb >= c)) continue;
                    const int id = (int)add_pt<TP_MIX>(pts, np, 2);
                    if (id < 0 || nfp >= FP_MIX) return 1;
                    const double t = __ddiv_rn(__dsub_rn(c, ga), __dsub_rn(gb, ga));
                    pts[id].p[a] = sd;
                    pts[id].p[along] = __dmul_rn(__dadd_rn((double)k, t), 0.5);
                    pts[id].p[across] = 0.5;
                    pts[id].key = gk_make(L0[0], L0[1], L0[2], (unsigned)along, (unsigned)(lvl + 1));
                    pw[id][a] = wlat(X, a, plane);
                    pw[id][along] = wfrac(X, along, 2 * C[along] + k, lvl + 1, t);
                    pw[id][across] = wlat(X, across, L0[across]);
                    fp[nfp++] = (signed char)id;
                }
            return 0;
        }
    }
    if (lvl > 0) {
        const int64_t Q[3] = {N[0] >> 1, N[1] >> 1, N[2] >> 1};
        const int64_t q = tri_cube_at(X, Q[0], Q[1], Q[2], lvl - 1);
        if (q < 0) return 0;
        double qu[2], qv[2];
        const int nn = cube_fold_roots(X, q, a, qu, qv);
        const int64_t su = C[ua] - 2 * Q[ua], sv = C[va] - 2 * Q[va];  // this face's quarter
        for (int r = 0; r < nn; r++) {
            if ((qu[r] >= 0.5) != (su == 1) || (qv[r] >= 0.5) != (sv == 1)) continue;
            const int id = (int)add_pt<TP_MIX>(pts, np, 2);
            if (id < 0 || nfp >= FP_MIX) return 1;
            pts[id].p[a] = sd;
            pts[id].p[ua] = __dsub_rn(__dmul_rn(2.0, qu[r]), (double)su);
            pts[id].p[va] = __dsub_rn(__dmul_rn(2.0, qv[r]), (double)sv);
            int64_t L[3] = {Q[0] * 2 * sc, Q[1] * 2 * sc, Q[2] * 2 * sc};
            L[a] = plane;
            pts[id].key = gk_make(L[0], L[1], L[2], 8u + 4u * a + 2u * (side_n == 0 ? 1u : 0u) + (unsigned)r,
                                  (unsigned)(lvl - 1));
            pw[id][a] = wlat(X, a, plane);
            pw[id][ua] = wfrac(X, ua, Q[ua], lvl - 1, qu[r]);
            pw[id][va] = wfrac(X, va, Q[va], lvl - 1, qv[r]);
            fp[nfp++] = (signed char)id;
        }
    }
    return 0;
}

// returns 0 on success, 1 on an inconsistency (cube skipped).  MIX: the cube
// has neighbours of another size (cubes of different sizes, section 2.3):
// halved edges take the crossing of the half where the sign changes; across
// a face with finer neighbours the face curve takes their fold ends and the
// points on the face's inner half-lines; across a face of a coarser
// neighbour it takes that cube's fold ends falling in this face.  Every
// point's world position is computed in the frame of the cube or edge it
// belongs to.
template <bool MIX>
__device__ int tri_cube(const TriCtx &X, int64_t ci, TriOut &o, unsigned long long *degen)
{
    constexpr int NP = MIX ? TP_MIX : TP_MAX;
    constexpr int FP = MIX ? FP_MIX : 4;
    uint64_t ck = X.cubes[ci];
    int lvl = (int)gk_level(ck);
    int64_t C[3] = {gk_x(ck), gk_y(ck), gk_z(ck)};
    int64_t sc = (int64_t)1 << (X.max_depth - lvl);
    double g[8];
    for (int v = 0; v < 8; v++) g[v] = X.phi[X.cvid[ci * 8 + v]];
    const double c = X.c;
    // inside bits, compared once: bit v = (g[v] >= c)
    int sg = 0;
    for (int v = 0; v < 8; v++) sg |= (g[v] >= c ? 1 : 0) << v;
    if (sg == 0 || sg == 0xFF) return 0;

    TPt pts[NP];
    double pw[MIX ? NP : 1][3];   // world coordinates (MIX)
    int np = 0;
    const bool fine_ok = MIX && lvl < X.max_depth;
    const int64_t s2 = sc >> 1;
    signed char eid[12];
    for (int a = 0; a < 3; a++) {
        int ua, va;
        axes_other(a, ua, va);
        for (int e = 0; e < 4; e++) {
            int o1 = e & 1, o2 = e >> 1;
            int b0[3], b1[3];
            b0[a] = 0; b1[a] = 1; b0[ua] = b1[ua] = o1; b0[va] = b1[va] = o2;
            const int v0 = b0[0] + 2 * b0[1] + 4 * b0[2], v1 = b1[0] + 2 * b1[1] + 4 * b1[2];
            eid[4 * a + e] = -1;
            if (((sg >> v0) & 1) == ((sg >> v1) & 1)) continue;
            double g0 = g[v0], g1 = g[v1];
            int id = (int)add_pt<NP>(pts, np, 0);
            int64_t L[3];
            L[a] = C[a] * sc; L[ua] = (C[ua] + o1) * sc; L[va] = (C[va] + o2) * sc;
            int64_t mid = -1;
            if (fine_ok) {
                int64_t Lm[3] = {L[0], L[1], L[2]};
                Lm[a] += s2;
                mid = tri_vert(X, Lm[0], Lm[1], Lm[2]);
            }
            if (MIX && mid >= 0) {
                // halved edge: the half where the sign changes
                const double gm = X.phi[mid];
                const int half = ((g0 >= c) == (gm >= c)) ? 1 : 0;
                const double ga = half ? gm : g0, gb = half ? g1 : gm;
                const double t = __ddiv_rn(__dsub_rn(c, ga), __dsub_rn(gb, ga));
                pts[id].p[a] = __dmul_rn(__dadd_rn((double)half, t), 0.5);
                L[a] += half * s2;
                pts[id].key = gk_make(L[0], L[1], L[2], (unsigned)a, (unsigned)(lvl + 1));
                if (MIX) pw[id][a] = wfrac(X, a, 2 * C[a] + half, lvl + 1, t);
            } else {
                pts[id].p[a] = __ddiv_rn(__dsub_rn(c, g0), __dsub_rn(g1, g0));
                pts[id].key = gk_make(L[0], L[1], L[2], (unsigned)a, (unsigned)lvl);
                if (MIX) pw[id][a] = wfrac(X, a, C[a], lvl, pts[id].p[a]);
            }
            pts[id].p[ua] = o1;
            pts[id].p[va] = o2;
            if (MIX) { pw[id][ua] = wlat(X, ua, L[ua]); pw[id][va] = wlat(X, va, L[va]); }
            eid[4 * a + e] = (signed char)id;
        }
    }
    // fold roots of this cube along each axis
    double rt[3][2][2];
    int nr[3];
    for (int a = 0; a < 3; a++) {
        double ru[2], rv[2];
        if (X.fcount) {
            nr[a] = X.fcount[ci * 4 + a];
            for (int r = 0; r < nr[a]; r++) {
                ru[r] = X.froot[ci * 12 + 4 * a + 2 * r];
                rv[r] = X.froot[ci * 12 + 4 * a + 2 * r + 1];
            }
        } else {
            nr[a] = fold_solve(g, a, c, ru, rv, 0.0, sg);
        }
        for (int r = 0; r < nr[a]; r++) { rt[a][r][0] = ru[r]; rt[a][r][1] = rv[r]; }
    }
    // critical points: an a-fold root and a b-fold root that share the third
    // axis' coordinate lie on crossing lines; the b-root takes the a-root's
    // value of that coordinate, so segments along each fold line are exactly
    // parallel to its axis (pairs in the order (0,1), (0,2), (1,2))
    signed char xa[12], xi[12], xb[12], xj[12];
    int nx = 0;
    for (int a = 0; a < 3; a++)
        for (int b = a + 1; b < 3; b++) {
            int cc = 3 - a - b;
            int ua, va, ub, vb;
            axes_other(a, ua, va);
            axes_other(b, ub, vb);
            for (int i = 0; i < nr[a]; i++)
                for (int j = 0; j < nr[b]; j++) {
                    double ca = rt[a][i][cc == ua ? 0 : 1], cb = rt[b][j][cc == ub ? 0 : 1];
                    if (fabs(ca - cb) > 1e-9) continue;
                    rt[b][j][cc == ub ? 0 : 1] = ca;
                    xa[nx] = (signed char)a; xi[nx] = (signed char)i; xb[nx] = (signed char)b; xj[nx] = (signed char)j;
                    nx++;
                }
        }
    // fold ends: own (both faces) and the same-size neighbours' ends on shared faces
    signed char fpt[6][FP];
    int nfp[6] = {0, 0, 0, 0, 0, 0};
    signed char fend[3][2][2];
    for (int a = 0; a < 3; a++) {
        int ua, va;
        axes_other(a, ua, va);
        for (int r = 0; r < nr[a]; r++) {
            for (int sd = 0; sd < 2; sd++) {
                int id = (int)add_pt<NP>(pts, np, 1);
                if (id < 0) return 1;
                pts[id].p[a] = sd; pts[id].p[ua] = rt[a][r][0]; pts[id].p[va] = rt[a][r][1];
                int64_t L[3] = {C[0] * sc, C[1] * sc, C[2] * sc};
                L[a] = (C[a] + sd) * sc;
                pts[id].key = gk_make(L[0], L[1], L[2], 8u + 4u * a + 2u * (sd == 0 ? 1u : 0u) + (unsigned)r, (unsigned)lvl);
                if (MIX)
                    for (int q = 0; q < 3; q++) pw[id][q] = wfrac(X, q, C[q], lvl, pts[id].p[q]);
                fend[a][r][sd] = (signed char)id;
                fpt[2 * a + sd][nfp[2 * a + sd]++] = (signed char)id;
            }
        }
        for (int sd = 0; sd < 2; sd++) {
            int nb = X.nbr[ci * 6 + 2 * a + sd];
            if (MIX && nb < 0) {
                if (tri_mixed_face(X, C, lvl, a, sd, fine_ok, pts, pw, np, fpt[2 * a + sd], nfp[2 * a + sd]))
                    return 1;
                continue;
            }
            if (nb < 0) continue;
            double nu_[2], nv_[2];
            int nn;
            if (X.fcount) {
                nn = X.fcount[(int64_t)nb * 4 + a];
                for (int r = 0; r < nn; r++) {
                    nu_[r] = X.froot[(int64_t)nb * 12 + 4 * a + 2 * r];
                    nv_[r] = X.froot[(int64_t)nb * 12 + 4 * a + 2 * r + 1];
                }
            } else {
                double gn[8];
                for (int v = 0; v < 8; v++) gn[v] = X.phi[X.cvid[(int64_t)nb * 8 + v]];
                nn = fold_solve(gn, a, c, nu_, nv_);
            }
            for (int r = 0; r < nn; r++) {
                int id = (int)add_pt<NP>(pts, np, 2);
                if (id < 0 || nfp[2 * a + sd] >= FP) return 1;
                pts[id].p[a] = sd; pts[id].p[ua] = nu_[r]; pts[id].p[va] = nv_[r];
                int64_t L[3] = {C[0] * sc, C[1] * sc, C[2] * sc};
                L[a] = (C[a] + sd) * sc;
                pts[id].key = gk_make(L[0], L[1], L[2], 8u + 4u * a + 2u * (sd == 1 ? 1u : 0u) + (unsigned)r, (unsigned)lvl);
                if (MIX)
                    for (int q = 0; q < 3; q++) pw[id][q] = wfrac(X, q, C[q], lvl, pts[id].p[q]);
                fpt[2 * a + sd][nfp[2 * a + sd]++] = (signed char)id;
            }
        }
    }
    signed char chain[3][2][4];
    int nch[3][2];
    for (int a = 0; a < 3; a++)
        for (int r = 0; r < nr[a]; r++) { chain[a][r][0] = fend[a][r][0]; nch[a][r] = 1; }
    for (int t = 0; t < nx; t++) {
        int a = xa[t], i = xi[t], b = xb[t], j = xj[t];
        int cc = 3 - a - b;
        int ua, va, ub, vb;
        axes_other(a, ua, va);
        axes_other(b, ub, vb);
        int id = (int)add_pt<NP>(pts, np, 3);
        if (id < 0) return 1;
        TPt &P = pts[id];
        P.p[a] = rt[b][j][a == ub ? 0 : 1];
        P.p[b] = rt[a][i][b == ua ? 0 : 1];
        P.p[cc] = rt[a][i][cc == ua ? 0 : 1];
        if (MIX)
            for (int q = 0; q < 3; q++) pw[id][q] = wfrac(X, q, C[q], lvl, P.p[q]);
        P.fa = (signed char)a; P.fb = (signed char)b;
        // dg/dx_cc at the point: the outward normal is -sign(dg/dx_cc) e_cc
        double dg = 0;
        for (int v = 0; v < 8; v++) {
            double f = 1.0;
            for (int q = 0; q < 3; q++) {
                int bit = (v >> q) & 1;
                f *= (q == cc) ? (bit ? 1.0 : -1.0) : (bit ? P.p[q] : 1.0 - P.p[q]);
            }
            dg += f * g[v];
        }
        bool cyclic = !(a == 0 && b == 2);   // (a,b,cc) an even permutation
        P.rh = (signed char)(cyclic == (dg < 0.0) ? 1 : 0);
        P.key = gk_make(C[0] * sc, C[1] * sc, C[2] * sc, 20u + 4u * (unsigned)(a + b - 1) + 2u * i + j, (unsigned)lvl);
        if (nch[a][i] < 3) chain[a][i][nch[a][i]++] = (signed char)id;
        if (nch[b][j] < 3) chain[b][j][nch[b][j]++] = (signed char)id;
    }
    for (int a = 0; a < 3; a++)
        for (int r = 0; r < nr[a]; r++) {
            signed char *ch = chain[a][r];
            int n = nch[a][r];
            if (n == 3 && pts[ch[2]].p[a] < pts[ch[1]].p[a]) { signed char t = ch[1]; ch[1] = ch[2]; ch[2] = t; }
            ch[n++] = fend[a][r][1];
            for (int k = 0; k + 1 < n; k++) {
                int p0 = ch[k], p1 = ch[k + 1];
                if (pts[p0].kind == 3) pts[p0].nb[pts[p0].fa == a ? 0 : 2] = (signed char)p1;
                else pts[p0].nb[0] = (signed char)p1;
                if (pts[p1].kind == 3) pts[p1].nb[pts[p1].fa == a ? 1 : 3] = (signed char)p0;
                else pts[p1].nb[0] = (signed char)p0;
            }
        }
    // face arcs -> successor along the loops
    signed char nxt[NP];
    for (int i = 0; i < np; i++) nxt[i] = -1;
    for (int a = 0; a < 3; a++) {
        int ua, va;
        axes_other(a, ua, va);
        for (int sd = 0; sd < 2; sd++) {
            double h[4];
            int fs = 0;
            for (int k = 0; k < 4; k++) {
                int b[3];
                b[a] = sd; b[ua] = k & 1; b[va] = k >> 1;
                const int vk = b[0] + 2 * b[1] + 4 * b[2];
                h[k] = g[vk];
                fs |= ((sg >> vk) & 1) << k;
            }
            // face edges in the (u,v) frame: 0 v=0, 1 u=1, 2 v=1, 3 u=0
            int ep[4];
            for (int e = 0; e < 4; e++) {
                int along = (e & 1) ? va : ua;
                int fixed = (e & 1) ? ua : va;
                int fval = (e == 1 || e == 2) ? 1 : 0;
                int bits[3];
                bits[along] = 0; bits[a] = sd; bits[fixed] = fval;
                int o1, o2;
                axes_other(along, o1, o2);
                ep[e] = eid[4 * along + bits[o1] + 2 * bits[o2]];
            }
            int around00;
            double us;
            int narc = face_arcs(h, c, around00, us, fs);
            int fid = 2 * a + sd;
            if (narc == 0) {
                if (nfp[fid] > 0) return 1;
                continue;
            }
            // start test: the curve leaves the boundary point into the face,
            // with the inside on its right seen from outside the cube.  With
            // hs = +-1 (sd ? 1 : -1)(a == 1 ? -1 : 1) the test values are
            // hs (h1 - h0), hs (h3 - h1), -hs (h3 - h2), -hs (h2 - h0); the
            // sign of a difference of doubles is that of their comparison
            const bool hp = (sd != 0) == (a != 1);
            auto st_pos = [&](int e) -> bool {
                switch (e) {
                case 0: return hp ? h[1] > h[0] : h[1] < h[0];
                case 1: return hp ? h[3] > h[1] : h[3] < h[1];
                case 2: return hp ? h[3] < h[2] : h[3] > h[2];
                default: return hp ? h[2] < h[0] : h[2] > h[0];
                }
            };
            int pr[2][2];
            if (narc == 1) {
                int k = 0;
                for (int e = 0; e < 4; e++)
                    if (ep[e] >= 0) { if (k < 2) pr[0][k] = e; k++; }
                if (k != 2) return 1;
            } else {
                if (around00) { pr[0][0] = 0; pr[0][1] = 3; pr[1][0] = 2; pr[1][1] = 1; }
                else { pr[0][0] = 0; pr[0][1] = 1; pr[1][0] = 2; pr[1][1] = 3; }
            }
            for (int ai = 0; ai < narc; ai++) {
                int e1 = pr[ai][0], e2 = pr[ai][1];
                if (ep[e1] < 0 || ep[e2] < 0) return 1;
                bool s1 = st_pos(e1), s2 = st_pos(e2);
                if (s1 == s2) return 1;
                int S = s1 ? ep[e1] : ep[e2], T = s1 ? ep[e2] : ep[e1];
                int mid[FP], nm = 0;
                for (int t = 0; t < nfp[fid]; t++) {
                    int id = fpt[fid][t];
                    if (narc == 2) {
                        bool low = pts[id].p[ua] < us;
                        bool arc_low = ai == 0 ? (around00 != 0) : (around00 == 0);
                        if (low != arc_low) continue;
                    }
                    mid[nm++] = id;
                }
                int ax = ua;
                double sg = 1.0;
                if (nm > 1) {
                    double du = pts[T].p[ua] - pts[S].p[ua], dv = pts[T].p[va] - pts[S].p[va];
                    ax = fabs(du) >= fabs(dv) ? ua : va;
                    sg = (ax == ua ? du : dv) >= 0 ? 1.0 : -1.0;
                }
                for (int i1 = 1; i1 < nm; i1++) {
                    int x = mid[i1], j = i1 - 1;
                    while (j >= 0) {
                        double kx = sg * pts[x].p[ax], kj = sg * pts[mid[j]].p[ax];
                        if (kj > kx || (kj == kx && pts[mid[j]].key > pts[x].key)) { mid[j + 1] = mid[j]; j--; }
                        else break;
                    }
                    mid[j + 1] = x;
                }
                int prev = S;
                for (int i1 = 0; i1 <= nm; i1++) {
                    int cur = i1 < nm ? mid[i1] : T;
                    if (nxt[prev] >= 0) return 1;
                    nxt[prev] = (signed char)cur;
                    prev = cur;
                }
            }
        }
    }
    for (int i = 0; i < np; i++)
        if (pts[i].kind != 3 && nxt[i] < 0) return 1;

    float pf[NP][3];
    for (int i = 0; i < np; i++)
        for (int a = 0; a < 3; a++) pf[i][a] = (float)pts[i].p[a];
    // pieces: faces of the graph of loops and fold segments, traced with the
    // face on the left; at a critical point take the next segment clockwise
    unsigned long long used_loop = 0ull;
    unsigned char used_fold[NP];
    for (int i = 0; i < np; i++) used_fold[i] = 0;
    const int cw_r[4] = {3, 2, 0, 1}, cw_l[4] = {2, 3, 1, 0};
    for (int i0 = 0; i0 < np; i0++) {
        if (pts[i0].kind == 3 || ((used_loop >> i0) & 1ull)) continue;
        unsigned char poly[POLY_MAX];
        int n = 0;
        int cur = i0, slot = -1;
        bool ok = true;
        for (int steps = 0;; steps++) {
            if (steps >= POLY_MAX || n >= POLY_MAX) { ok = false; break; }
            poly[n++] = (unsigned char)cur;
            int nx;
            if (slot < 0) { used_loop |= 1ull << cur; nx = nxt[cur]; }
            else { used_fold[cur] |= (unsigned char)(1u << slot); nx = pts[cur].nb[slot]; }
            if (nx < 0) { ok = false; break; }
            int ns;
            if (slot < 0) ns = pts[nx].kind == 1 ? 0 : -1;
            else if (pts[nx].kind != 3) ns = -1;
            else {
                int back = -1;
                for (int k = 0; k < 4; k++) if (pts[nx].nb[k] == cur) back = k;
                if (back < 0) { ok = false; break; }
                ns = pts[nx].rh ? cw_r[back] : cw_l[back];
                if (pts[nx].nb[ns] < 0) { ok = false; break; }
            }
            cur = nx;
            slot = ns;
            if (slot < 0 && cur == i0) break;
            if (slot < 0 && ((used_loop >> cur) & 1ull)) { ok = false; break; }
            if (slot >= 0 && ((used_fold[cur] >> slot) & 1u)) { ok = false; break; }
        }
        if (!ok) return 1;
        if (n >= 3) clip_piece(pts, pf, poly, n, o, degen);
    }
    // points in world coordinates
    if (MIX && np <= o.pt_cap) {
        for (int i = 0; i < np; i++) {
            double *dst = o.pt_xyz + 3 * (o.pt_off + i);
            for (int a = 0; a < 3; a++) dst[a] = pw[i][a];
            o.pt_keys[o.pt_off + i] = pts[i].key;
        }
    } else if (np <= o.pt_cap) {
        double h = ldexp(X.min_edge, X.max_depth - lvl);
        double lo[3], hi[3];
        for (int a = 0; a < 3; a++) {
            lo[a] = __dadd_rn(X.origin[a], __dmul_rn((double)(C[a] * sc), X.min_edge));
            hi[a] = __dadd_rn(X.origin[a], __dmul_rn((double)((C[a] + 1) * sc), X.min_edge));
        }
        for (int i = 0; i < np; i++) {
            double *dst = o.pt_xyz + 3 * (o.pt_off + i);
            for (int a = 0; a < 3; a++) {
                // the cube's own faces (local 0 or 1, read from the bits)
                // take the lattice coordinates; lo + (-0) h is lo as well
                double f = pts[i].p[a];
                const unsigned long long fb = (unsigned long long)__double_as_longlong(f);
                if ((fb << 1) == 0ull) dst[a] = lo[a];
                else if (fb == 0x3FF0000000000000ull) dst[a] = hi[a];
                else dst[a] = __dadd_rn(lo[a], __dmul_rn(f, h));
            }
            o.pt_keys[o.pt_off + i] = pts[i].key;
        }
    }
    o.npt = np;
    return 0;
}

// both faces normal to axis a are cut by the surface (needed for a fold root)
__device__ __forceinline__ bool fold_faces_straddle(int sg, int a)
{
    int ua, va;
    axes_other(a, ua, va);
    int nlo = 0, nup = 0;
    for (int k = 0; k < 4; k++) {
        int b[3];
        b[a] = 0; b[ua] = k & 1; b[va] = k >> 1;
        nlo += (sg >> (b[0] + 2 * b[1] + 4 * b[2])) & 1;
        b[a] = 1;
        nup += (sg >> (b[0] + 2 * b[1] + 4 * b[2])) & 1;
    }
    return nlo != 0 && nlo != 4 && nup != 0 && nup != 4;
}

// FP32 screen for the fold roots of axis a: false only when the quadratic
// in u certainly has no root in (0,1) (its FP32 coefficients are within
// ~1e-6 of their size; the margins below are 1e-3 of it), so the FP64
// solver runs only where it may find a root
__device__ __forceinline__ bool fold_may_have_roots(const float *gc, int a)
{
    int ua, va;
    axes_other(a, ua, va);
    float lo[4], up[4];
    for (int k = 0; k < 4; k++) {
        int b[3];
        b[a] = 0; b[ua] = k & 1; b[va] = k >> 1;
        lo[k] = gc[b[0] + 2 * b[1] + 4 * b[2]];
        b[a] = 1;
        up[k] = gc[b[0] + 2 * b[1] + 4 * b[2]];
    }
    const float p0 = lo[0], p1 = lo[1] - lo[0], p2 = lo[2] - lo[0], p3 = lo[3] - lo[1] - lo[2] + lo[0];
    const float d0 = up[0] - lo[0], d1 = up[1] - lo[1], d2 = up[2] - lo[2], d3 = up[3] - lo[3];
    const float q0 = d0, q1 = d1 - d0, q2 = d2 - d0, q3 = d3 - d1 - d2 + d0;
    const float A2 = p1 * q3 - p3 * q1, A1 = p0 * q3 + p1 * q2 - p2 * q1 - p3 * q0, A0 = p0 * q2 - p2 * q0;
    const float mag = fabsf(p1 * q3) + fabsf(p3 * q1) + fabsf(p0 * q3) + fabsf(p1 * q2) + fabsf(p2 * q1) +
                      fabsf(p3 * q0) + fabsf(p0 * q2) + fabsf(p2 * q0);
    if (!(mag > 1e-30f)) return true;                      // degenerate: let FP64 decide
    if (fabsf(A2) <= 1e-3f * mag) return true;             // near linear
    const float disc = A1 * A1 - 4.f * A2 * A0, scale = A1 * A1 + 4.f * fabsf(A2 * A0);
    if (disc < -1e-3f * scale) return false;               // no real root
    if (disc <= 1e-3f * scale) return true;                // near a double root
    const float sq = sqrtf(disc), w = A1 >= 0.f ? -0.5f * (A1 + sq) : -0.5f * (A1 - sq);
    if (w == 0.f) return true;
    const float u1 = w / A2, u2 = A0 / w;
    return (u1 > -0.01f && u1 < 1.01f) || (u2 > -0.01f && u2 < 1.01f);
}

// fold roots of every cube (own ends and, across faces, the neighbours'
// ends are read from this table instead of being solved again)
__global__ void __launch_bounds__(128) k_fold_table(TriCtx X, uint8_t *__restrict__ fcount, double *__restrict__ froot)
{
    int64_t ci = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= X.ncubes) return;
    double g[8];
    for (int v = 0; v < 8; v++) g[v] = X.phi[X.cvid[ci * 8 + v]];
    int sg = 0;
    float gc[8];
    for (int v = 0; v < 8; v++) {
        sg |= (g[v] >= X.c ? 1 : 0) << v;
        gc[v] = (float)(g[v] - X.c);
    }
    uint32_t cnt = 0;
    for (int a = 0; a < 3 && sg != 0 && sg != 0xFF; a++) {
        double ru[2], rv[2];
        int nr = fold_faces_straddle(sg, a) && fold_may_have_roots(gc, a) ? fold_solve(g, a, X.c, ru, rv, 0.0, sg) : 0;
        cnt |= (uint32_t)nr << (8 * a);
        for (int r = 0; r < nr; r++) {
            froot[ci * 12 + 4 * a + 2 * r] = ru[r];
            froot[ci * 12 + 4 * a + 2 * r + 1] = rv[r];
        }
    }
    *reinterpret_cast<uint32_t *>(fcount + ci * 4) = cnt;
}

// The same table in two passes: an FP32 screen over every cube lists the
// (cube, axis) pairs whose fold roots may exist and zeroes every count; the
// FP64 solver then runs over the list in full warps (a warp of the one-pass
// kernel runs the solver whenever any of its cubes needs it).  List entry:
// cube << 2 | axis.
__global__ void __launch_bounds__(256) k_fold_screen(TriCtx X, uint8_t *__restrict__ fcount,
                                                     uint32_t *__restrict__ list, unsigned *nlist)
{
    const int64_t ci = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned need = 0;
    if (ci < X.ncubes) {
        int sg = 0;
        float gc[8];
        for (int v = 0; v < 8; v++) {
            const double g = X.phi[X.cvid[ci * 8 + v]];
            sg |= (g >= X.c ? 1 : 0) << v;
            gc[v] = (float)(g - X.c);
        }
        if (sg != 0 && sg != 0xFF)
            for (int a = 0; a < 3; a++)
                if (fold_faces_straddle(sg, a) && fold_may_have_roots(gc, a)) need |= 1u << a;
        *reinterpret_cast<uint32_t *>(fcount + ci * 4) = 0u;
    }
    const unsigned lane = threadIdx.x & 31;
    const unsigned cntv = (unsigned)__popc(need);
    unsigned incl = cntv;
    for (int o = 1; o < 32; o <<= 1) {
        const unsigned t = __shfl_up_sync(0xffffffffu, incl, o);
        if (lane >= (unsigned)o) incl += t;
    }
    const unsigned tot = __shfl_sync(0xffffffffu, incl, 31);
    if (tot == 0) return;
    unsigned base = 0;
    if (lane == 31) base = atomicAdd(nlist, tot);
    base = __shfl_sync(0xffffffffu, base, 31);
    unsigned pos = base + incl - cntv;
    for (int a = 0; a < 3; a++)
        if ((need >> a) & 1u) list[pos++] = ((uint32_t)ci << 2) | (uint32_t)a;
}

__global__ void __launch_bounds__(128) k_fold_solve(TriCtx X, const uint32_t *__restrict__ list,
                                                    const unsigned *__restrict__ nlist, uint8_t *__restrict__ fcount,
                                                    double *__restrict__ froot)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= (int64_t)*nlist) return;
    const uint32_t e = list[t];
    const int64_t ci = (int64_t)(e >> 2);
    const int a = (int)(e & 3u);
    double g[8];
    int sg = 0;
    for (int v = 0; v < 8; v++) {
        g[v] = X.phi[X.cvid[ci * 8 + v]];
        sg |= (g[v] >= X.c ? 1 : 0) << v;
    }
    double ru[2], rv[2];
    const int nr = fold_solve(g, a, X.c, ru, rv, 0.0, sg);
    fcount[ci * 4 + a] = (uint8_t)nr;
    for (int r = 0; r < nr; r++) {
        froot[ci * 12 + 4 * a + 2 * r] = ru[r];
        froot[ci * 12 + 4 * a + 2 * r + 1] = rv[r];
    }
}

// first pass: trace every cube, count its output and stage it when it fits
// Cube classes for the tracing order: cubes of one class take the same
// branches (which edges cross, how many fold roots, how many faces carry a
// neighbour's fold ends; for the marks, which run before the fold table,
// how many axes the FP32 fold screen leaves open), so warps diverge less.  Class 1024 * min(faces
// whose neighbour has fold roots on the shared axis, 3) + 256 * min(roots,
// 3) + the corner sign pattern; cubes without a surface go last.
#define TRI_CLASSES 4097
static_assert(1024 * 3 + 256 * 3 + 255 < TRI_CLASSES - 1, "surface classes stay below the last (no surface)");
__global__ void k_tri_class(TriCtx X, int32_t *__restrict__ cls, unsigned *__restrict__ hist)
{
    __shared__ unsigned sh[TRI_CLASSES];
    for (int k = threadIdx.x; k < TRI_CLASSES; k += blockDim.x) sh[k] = 0;
    __syncthreads();
    int64_t ci = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ci < X.ncubes) {
        int sg = 0;
        double g[8];
        for (int v = 0; v < 8; v++) {
            g[v] = X.phi[X.cvid[ci * 8 + v]];
            sg |= (g[v] >= X.c ? 1 : 0) << v;
        }
        int k = TRI_CLASSES - 1;
        if (sg != 0 && sg != 0xFF) {
            int nr = 0, nbf = 0;
            if (!X.fcount) {
                // before the fold table (the marks): the axes whose fold
                // quadratic the FP32 screen cannot rule out
                float gc[8];
                for (int v = 0; v < 8; v++) gc[v] = (float)(g[v] - X.c);
                for (int a = 0; a < 3; a++)
                    if (fold_faces_straddle(sg, a) && fold_may_have_roots(gc, a)) nr++;
            } else {
                uint32_t f = *reinterpret_cast<const uint32_t *>(X.fcount + ci * 4);
                nr = (int)(f & 0xFF) + (int)((f >> 8) & 0xFF) + (int)((f >> 16) & 0xFF);
                if (X.nbr)
                    for (int fc = 0; fc < 6; fc++) {
                        const int nb = X.nbr[ci * 6 + fc];
                        if (nb >= 0 && X.fcount[(int64_t)nb * 4 + (fc >> 1)]) nbf++;
                    }
            }
            k = 1024 * (nbf < 3 ? nbf : 3) + 256 * (nr < 3 ? nr : 3) + sg;
        }
        cls[ci] = k;
        atomicAdd(&sh[k], 1u);
    }
    __syncthreads();
    for (int k = threadIdx.x; k < TRI_CLASSES; k += blockDim.x)
        if (sh[k]) atomicAdd(&hist[k], sh[k]);
}

// order[pos] = cube: classes in turn (any order within a class).  Each block
// counts its cubes per class in shared memory and reserves one range per
// class with a single global atomic.
__global__ void k_tri_order(const int32_t *__restrict__ cls, int64_t n, unsigned *__restrict__ cursor,
                            int32_t *__restrict__ order)
{
    __shared__ unsigned cnt[TRI_CLASSES], base[TRI_CLASSES];
    for (int k = threadIdx.x; k < TRI_CLASSES; k += blockDim.x) cnt[k] = 0;
    __syncthreads();
    int64_t ci = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    int k = -1;
    unsigned local = 0;
    if (ci < n) {
        k = cls[ci];
        local = atomicAdd(&cnt[k], 1u);
    }
    __syncthreads();
    for (int q = threadIdx.x; q < TRI_CLASSES; q += blockDim.x)
        if (cnt[q]) base[q] = atomicAdd(&cursor[q], cnt[q]);
    __syncthreads();
    if (k >= 0) order[base[k] + local] = (int32_t)ci;
}

// cubes grouped by class (order, n entries; nullptr when it cannot be
// built, and then *n_surf = n); the first *n_surf have a surface
static int tri_order(const TriCtx &X, int32_t **d_order, int64_t *n_surf, cudaStream_t st)
{
    const int64_t n = X.ncubes;
    *d_order = nullptr;
    *n_surf = n;
    if (n <= 0 || n >= ((int64_t)1 << 31)) return GS_OK;
    int32_t *cls = nullptr, *order = nullptr;
    unsigned *hist = nullptr;
    if (gs_alloc((void **)&cls, sizeof(int32_t) * (size_t)n, st) ||
        gs_alloc((void **)&order, sizeof(int32_t) * (size_t)n, st) ||
        gs_alloc((void **)&hist, sizeof(unsigned) * TRI_CLASSES, st)) {
        cudaGetLastError();
        gs_free(cls, st); gs_free(order, st); gs_free(hist, st);
        return GS_OK;   // trace in cube order
    }
    const unsigned nb = (unsigned)((n + 127) / 128);
    cudaMemsetAsync(hist, 0, sizeof(unsigned) * TRI_CLASSES, st);
    GS_LAUNCH(k_tri_class, nb, 128, 0, st)(X, cls, hist);
    unsigned hh[TRI_CLASSES];
    cudaError_t e = cudaMemcpyAsync(hh, hist, sizeof(hh), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = gs_sync(st);
    if (e != cudaSuccess) {
        gs_free(cls, st); gs_free(order, st); gs_free(hist, st);
        return gs_fail_cuda(e, "cube classes", __FILE__, __LINE__);
    }
    unsigned acc = 0;
    for (int k = 0; k < TRI_CLASSES; k++) { unsigned c = hh[k]; hh[k] = acc; acc += c; }
    cudaMemcpyAsync(hist, hh, sizeof(hh), cudaMemcpyHostToDevice, st);
    GS_LAUNCH(k_tri_order, nb, 128, 0, st)(cls, n, hist, order);
    gs_free(cls, st);
    gs_free(hist, st);
    *d_order = order;
    *n_surf = (int64_t)hh[TRI_CLASSES - 1];
    return GS_OK;
}

// MIX: over the list of cubes with neighbours of another size (count only);
// otherwise over all cubes, skipping those
template <bool MIX>
__global__ void __launch_bounds__(128) k_tri_count(TriCtx X, int64_t n_trace, int64_t *__restrict__ ntri,
                                                   int64_t *__restrict__ npt,
                                                   unsigned long long *errs, unsigned long long *surface,
                                                   uint64_t *st_tri, uint64_t *st_pk, double *st_xyz,
                                                   unsigned long long *degen, const int32_t *__restrict__ order,
                                                   const int64_t *__restrict__ mlist, const unsigned long long *nmlist)
{
    int64_t ci = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (MIX) {
        if (ci >= (int64_t)*nmlist) return;
        ci = mlist[ci];
        st_tri = nullptr;
    } else {
        if (ci >= n_trace) return;
        if (order) ci = order[ci];
        if (X.mixed && X.mixed[ci]) return;
    }
    TriOut o;
    o.ntri = 0; o.npt = 0;
    o.tri_keys = st_tri; o.pt_keys = st_pk; o.pt_xyz = st_xyz;
    o.tri_off = ci * TRI_STAGE_T; o.pt_off = ci * TRI_STAGE_P;
    o.tri_cap = st_tri ? TRI_STAGE_T : 0;
    o.pt_cap = st_tri ? TRI_STAGE_P : -1;
    int bad = tri_cube<MIX>(X, ci, o, st_tri ? degen : nullptr);
    if (bad) { atomicAdd(errs, 1ull); o.ntri = 0; o.npt = 0; }
    {
        // one atomic per warp for the surface-cube count
        const unsigned act = __activemask(), bal = __ballot_sync(act, o.npt > 0);
        if ((int)(threadIdx.x & 31) == __ffs(act) - 1 && bal) atomicAdd(surface, (unsigned long long)__popc(bal));
    }
    ntri[ci] = o.ntri;
    npt[ci] = o.npt;
}

// copy the k-th element (of a warp's concatenated per-lane runs of len
// elements, excl the exclusive prefix) from src_base + local to dst_base +
// local, lane by lane over the total: consecutive lanes write consecutive
// destination elements within a run
template <typename T>
__device__ __forceinline__ void warp_copy_runs(int len, int excl, int total, int lane, int64_t src_base,
                                               int64_t dst_base, const T *__restrict__ src, T *__restrict__ dst)
{
    const unsigned full = 0xffffffffu;
    for (int g0 = 0; g0 < total; g0 += 32) {
        const int g = g0 + lane;
        int owner = 0;   // the last lane whose run starts at or before g
#pragma unroll
        for (int step = 16; step > 0; step >>= 1) {
            const int e = __shfl_sync(full, excl, owner + step);
            if (e <= g) owner += step;
        }
        const int oe = __shfl_sync(full, excl, owner);
        const int64_t sb = __shfl_sync(full, src_base, owner), db = __shfl_sync(full, dst_base, owner);
        if (g < total) dst[db + (g - oe)] = src[sb + (g - oe)];
    }
    (void)len;
}

// staged cubes: copy to the scanned offsets, a warp's 32 cubes together
// (coalesced stores); the others go to the list of cubes traced again by
// k_tri_emit
__global__ void __launch_bounds__(128) k_tri_copy(int64_t n, const int64_t *__restrict__ tri_off,
                                                  const int64_t *__restrict__ pt_off, const uint64_t *__restrict__ st_tri,
                                                  const uint64_t *__restrict__ st_pk, const double *__restrict__ st_xyz,
                                                  uint64_t *__restrict__ tri_keys, uint64_t *__restrict__ pt_keys,
                                                  double *__restrict__ pt_xyz, int64_t *__restrict__ redo,
                                                  unsigned long long *nredo, const uint8_t *__restrict__ mixed)
{
    const unsigned full = 0xffffffffu;
    const int64_t ci = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const int lane = threadIdx.x & 31;
    bool over = false;
    int nt = 0, np = 0;
    int64_t t0 = 0, p0 = 0;
    if (ci < n && !(mixed && mixed[ci])) {
        t0 = tri_off[ci];
        p0 = pt_off[ci];
        const int64_t ntl = tri_off[ci + 1] - t0, npl = pt_off[ci + 1] - p0;
        if (ntl > TRI_STAGE_T || npl > TRI_STAGE_P) over = true;
        else { nt = (int)ntl; np = (int)npl; }
    }
    // runs per lane: 3 nt triangle keys, np point keys, 3 np coordinates
    int it = 3 * nt, ip = np;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const int vt = __shfl_up_sync(full, it, o), vp = __shfl_up_sync(full, ip, o);
        if (lane >= o) { it += vt; ip += vp; }
    }
    const int tt = __shfl_sync(full, it, 31), tp = __shfl_sync(full, ip, 31);
    const int et = it - 3 * nt, ep = ip - np;
    warp_copy_runs<uint64_t>(3 * nt, et, tt, lane, 3 * ci * TRI_STAGE_T, 3 * t0, st_tri, tri_keys);
    warp_copy_runs<uint64_t>(np, ep, tp, lane, ci * TRI_STAGE_P, p0, st_pk, pt_keys);
    warp_copy_runs<double>(3 * np, 3 * ep, 3 * tp, lane, 3 * ci * TRI_STAGE_P, 3 * p0, st_xyz, pt_xyz);
    const unsigned bal = __ballot_sync(full, over);
    if (!bal) return;
    unsigned long long base = 0;
    if (lane == 0) base = atomicAdd(nredo, (unsigned long long)__popc(bal));
    base = __shfl_sync(full, base, 0);
    if (over) redo[base + __popc(bal & ((1u << lane) - 1u))] = ci;
}

// final pass over the listed cubes (all cubes when list is null); MIX: the
// cubes with neighbours of another size, which the other passes skip
template <bool MIX>
__global__ void __launch_bounds__(128) k_tri_emit(TriCtx X, const int64_t *__restrict__ tri_off,
                                                  const int64_t *__restrict__ pt_off, uint64_t *__restrict__ tri_keys,
                                                  uint64_t *__restrict__ pt_keys, double *__restrict__ pt_xyz,
                                                  unsigned long long *degen, const int64_t *__restrict__ list,
                                                  const unsigned long long *nlist)
{
    int64_t ci = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (list) {
        if (ci >= (int64_t)*nlist) return;
        ci = list[ci];
    } else if (ci >= X.ncubes) {
        return;
    }
    if (!MIX && X.mixed && X.mixed[ci]) return;
    if (tri_off[ci + 1] == tri_off[ci] && pt_off[ci + 1] == pt_off[ci]) return;
    TriOut o;
    o.ntri = 0; o.npt = 0; o.tri_off = tri_off[ci]; o.pt_off = pt_off[ci];
    o.tri_cap = 1 << 30; o.pt_cap = 1 << 30;
    o.tri_keys = tri_keys; o.pt_keys = pt_keys; o.pt_xyz = pt_xyz;
    tri_cube<MIX>(X, ci, o, degen);
}

// list of the cubes flagged mixed (any order)
__global__ void k_mixed_list(const uint8_t *__restrict__ mixed, int64_t n, int64_t *__restrict__ list,
                             unsigned long long *nlist)
{
    const int64_t ci = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ci < n && mixed[ci]) list[atomicAdd(nlist, 1ull)] = ci;
}

// ---------------------------------------------------------------- host
int gs_triangulate(const TriCtx &X0, uint64_t **d_tri_keys, int64_t *ntri_total, uint64_t **d_pt_keys,
                   double **d_pt_xyz, int64_t *npt_total, unsigned long long *d_counters, cudaStream_t st)
{
    TriCtx X = X0;
    int64_t n = X.ncubes;
    *d_tri_keys = nullptr; *d_pt_keys = nullptr; *d_pt_xyz = nullptr;
    *ntri_total = 0; *npt_total = 0;
    if (n <= 0) return GS_OK;
    int64_t *ntri = nullptr, *npt = nullptr, *tot = nullptr;
    int rc = gs_alloc((void **)&ntri, sizeof(int64_t) * (size_t)(n + 1), st);
    if (!rc) rc = gs_alloc((void **)&npt, sizeof(int64_t) * (size_t)(n + 1), st);
    if (!rc) rc = gs_alloc((void **)&tot, 2 * sizeof(int64_t), st);
    if (rc) { gs_free(ntri, st); gs_free(npt, st); gs_free(tot, st); return rc; }
    // staging slots; without room for them every cube is traced twice
    uint64_t *st_tri = nullptr, *st_pk = nullptr;
    double *st_xyz = nullptr;
    if (cudaMallocAsync((void **)&st_tri, sizeof(uint64_t) * 3 * TRI_STAGE_T * (size_t)n, st) != cudaSuccess ||
        cudaMallocAsync((void **)&st_pk, sizeof(uint64_t) * TRI_STAGE_P * (size_t)n, st) != cudaSuccess ||
        cudaMallocAsync((void **)&st_xyz, sizeof(double) * 3 * TRI_STAGE_P * (size_t)n, st) != cudaSuccess) {
        cudaGetLastError();
        gs_free(st_tri, st); gs_free(st_pk, st); gs_free(st_xyz, st);
        st_tri = nullptr; st_pk = nullptr; st_xyz = nullptr;
    }
    unsigned nb = (unsigned)((n + 127) / 128);
    // fold-root table; without room for it each cube solves its neighbours' roots
    uint8_t *fcount = nullptr;
    double *froot = nullptr;
    if (cudaMallocAsync((void **)&fcount, 4 * (size_t)n, st) != cudaSuccess ||
        cudaMallocAsync((void **)&froot, sizeof(double) * 12 * (size_t)n, st) != cudaSuccess) {
        cudaGetLastError();
        gs_free(fcount, st); gs_free(froot, st);
        fcount = nullptr; froot = nullptr;
    } else {
        uint32_t *flist = nullptr;
        unsigned *nflist = nullptr;
        const bool screened = n < ((int64_t)1 << 30) &&
                              cudaMallocAsync((void **)&flist, sizeof(uint32_t) * 3 * (size_t)n, st) == cudaSuccess &&
                              cudaMallocAsync((void **)&nflist, sizeof(unsigned), st) == cudaSuccess;
        if (screened) {
            cudaMemsetAsync(nflist, 0, sizeof(unsigned), st);
            GS_LAUNCH(k_fold_screen, (unsigned)((n + 255) / 256), 256, 0, st)(X, fcount, flist, nflist);
            GS_LAUNCH(k_fold_solve, (unsigned)((3 * n + 127) / 128), 128, 0, st)(X, flist, nflist, fcount, froot);
        } else {
            cudaGetLastError();
            GS_LAUNCH(k_fold_table, nb, 128, 0, st)(X, fcount, froot);
        }
        gs_free(flist, st);
        gs_free(nflist, st);
        X.fcount = fcount;
        X.froot = froot;
    }
    cudaMemsetAsync(ntri + n, 0, sizeof(int64_t), st);
    cudaMemsetAsync(npt + n, 0, sizeof(int64_t), st);
    // tracing order by cube class (fewer divergent branches per warp); the
    // cubes without a surface come last and are not traced
    int32_t *order = nullptr;
    int64_t n_trace = n;
    rc = tri_order(X, &order, &n_trace, st);
    if (rc) {
        gs_free(ntri, st); gs_free(npt, st); gs_free(tot, st);
        gs_free(st_tri, st); gs_free(st_pk, st); gs_free(st_xyz, st);
        gs_free(fcount, st); gs_free(froot, st);
        return rc;
    }
    if (order) {
        cudaMemsetAsync(ntri, 0, sizeof(int64_t) * (size_t)n, st);
        cudaMemsetAsync(npt, 0, sizeof(int64_t) * (size_t)n, st);
    }
    if (n_trace > 0)
        GS_LAUNCH(k_tri_count<false>, (unsigned)((n_trace + 127) / 128), 128, 0, st)(
            X, n_trace, ntri, npt, d_counters + 0, d_counters + 2, st_tri, st_pk, st_xyz, d_counters + 1, order,
            nullptr, nullptr);
    int64_t *mlist = nullptr;
    unsigned long long *nmlist = nullptr;
    if (X.mixed) {
        rc = gs_alloc((void **)&mlist, sizeof(int64_t) * (size_t)n, st);
        if (!rc) rc = gs_alloc((void **)&nmlist, sizeof(unsigned long long), st);
        if (!rc) {
            cudaMemsetAsync(nmlist, 0, sizeof(unsigned long long), st);
            GS_LAUNCH(k_mixed_list, (unsigned)((n + 255) / 256), 256, 0, st)(X.mixed, n, mlist, nmlist);
            GS_LAUNCH(k_tri_count<true>, nb, 128, 0, st)(X, n, ntri, npt, d_counters + 0, d_counters + 2, nullptr,
                                                        nullptr, nullptr, d_counters + 1, nullptr, mlist, nmlist);
        }
    }
    gs_free(order, st);
    rc = gs_scan_i64(ntri, n + 1, tot, st);
    if (!rc) rc = gs_scan_i64(npt, n + 1, tot + 1, st);
    int64_t h[2] = {0, 0};
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(h, tot, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = gs_sync(st);
        if (e != cudaSuccess) rc = gs_fail_cuda(e, "triangle counts", __FILE__, __LINE__);
    }
    if (!rc) {
        rc = gs_alloc((void **)d_tri_keys, sizeof(uint64_t) * 3 * (size_t)(h[0] + 1), st);
        if (!rc) rc = gs_alloc((void **)d_pt_keys, sizeof(uint64_t) * (size_t)(h[1] + 1), st);
        if (!rc) rc = gs_alloc((void **)d_pt_xyz, sizeof(double) * 3 * (size_t)(h[1] + 1), st);
    }
    if (!rc && st_tri) {
        int64_t *redo = nullptr;
        unsigned long long *nredo = nullptr;
        rc = gs_alloc((void **)&redo, sizeof(int64_t) * (size_t)n, st);
        if (!rc) rc = gs_alloc((void **)&nredo, sizeof(unsigned long long), st);
        if (!rc) {
            cudaMemsetAsync(nredo, 0, sizeof(unsigned long long), st);
            GS_LAUNCH(k_tri_copy, nb, 128, 0, st)(n, ntri, npt, st_tri, st_pk, st_xyz, *d_tri_keys, *d_pt_keys,
                                                 *d_pt_xyz, redo, nredo, X.mixed);
            GS_LAUNCH(k_tri_emit<false>, nb, 128, 0, st)(X, ntri, npt, *d_tri_keys, *d_pt_keys, *d_pt_xyz, nullptr,
                                                        redo, nredo);
        }
        gs_free(redo, st); gs_free(nredo, st);
    } else if (!rc) {
        GS_LAUNCH(k_tri_emit<false>, nb, 128, 0, st)(X, ntri, npt, *d_tri_keys, *d_pt_keys, *d_pt_xyz, d_counters + 1,
                                                    nullptr, nullptr);
    }
    if (!rc && X.mixed)
        GS_LAUNCH(k_tri_emit<true>, nb, 128, 0, st)(X, ntri, npt, *d_tri_keys, *d_pt_keys, *d_pt_xyz, d_counters + 1,
                                                   mlist, nmlist);
    gs_free(mlist, st); gs_free(nmlist, st);
    gs_free(st_tri, st); gs_free(st_pk, st); gs_free(st_xyz, st);
    gs_free(fcount, st); gs_free(froot, st);
    gs_free(ntri, st); gs_free(npt, st); gs_free(tot, st);
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    *ntri_total = h[0];
    *npt_total = h[1];
    return GS_OK;
}

// ---------------------------------------------------------------- mixed precision marks
// For a surface cube with FP32 corner values g and bounds e: an edge point at
// t = (c - g0) / (g1 - g0) moves by at most h ((1 - t) e0 + t e1) / |g1 - g0|
// (first order); a face's saddle
// decision is safe when |h_s - c| exceeds the bound carried through h_s; a
// fold root (extreme and critical points) moves by at most the first-order
// bound from the root's derivative.  Where any bound exceeds tol the corners
// involved (all eight for a fold) are re-evaluated in FP64.
// in_list or order (nullable): only the n_in listed cubes; out_list
// (nullable): the cubes that marked a corner are appended to it
__global__ void __launch_bounds__(128) k_tri_marks(TriCtx X, const float *__restrict__ err, double tol,
                                                   int64_t *__restrict__ mark, unsigned long long *why,
                                                   const int64_t *__restrict__ in_list,
                                                   const int32_t *__restrict__ order, int64_t n_in,
                                                   int64_t *__restrict__ out_list, unsigned long long *n_out)
{
    int64_t ci = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (ci >= n_in) return;
    if (in_list) ci = in_list[ci];
    else if (order) ci = order[ci];
    uint64_t ck = X.cubes[ci];
    int lvl = (int)gk_level(ck);
    const float h = (float)ldexp(X.min_edge, X.max_depth - lvl);
    double g[8];
    float gc[8], e[8];
    int vid[8];
    const double c = X.c;
    int sg = 0;
    for (int v = 0; v < 8; v++) {
        vid[v] = X.cvid[ci * 8 + v];
        g[v] = X.phi[vid[v]];
        e[v] = err[vid[v]];
        gc[v] = (float)(g[v] - c);
        sg |= (g[v] >= c ? 1 : 0) << v;
    }
    if (sg == 0 || sg == 0xFF) return;
    // The bounds below are first-order estimates evaluated in FP32 from the
    // corner values minus c; they are inflated by 1% (and tol lowered by
    // 0.1%) so that their own rounding only ever marks more corners.
    const float tolf = (float)tol * 0.999f, infl = 1.01f;
    bool all = false, r_edge = false, r_face = false, r_fold = false;
    unsigned m = 0;
    for (int a = 0; a < 3 && !all; a++) {
        int ua, va;
        axes_other(a, ua, va);
        for (int k = 0; k < 4; k++) {
            int b0[3], b1[3];
            b0[a] = 0; b1[a] = 1; b0[ua] = b1[ua] = k & 1; b0[va] = b1[va] = k >> 1;
            int v0 = b0[0] + 2 * b0[1] + 4 * b0[2], v1 = b1[0] + 2 * b1[1] + 4 * b1[2];
            if (((sg >> v0) & 1) == ((sg >> v1) & 1)) continue;
            // t = (c - g0) / (g1 - g0) moves by ((1 - t) e0 + t e1) / |g1 - g0|
            // to first order; an FP64 corner has no error: re-evaluate the
            // larger contributor, and the other one if it alone exceeds the bound
            float dg = fabsf(gc[v1] - gc[v0]), t = fminf(fabsf(gc[v0]) / dg, 1.f);
            const float c0 = infl * h * (1.f - t) * e[v0], c1 = infl * h * t * e[v1], lim = tolf * dg;
            if (c0 + c1 > lim) {
                const int big = c0 >= c1 ? v0 : v1, small = c0 >= c1 ? v1 : v0;
                m |= 1u << big;
                if (fminf(c0, c1) > lim) m |= 1u << small;
                r_edge = true;
            }
        }
        for (int sd = 0; sd < 2; sd++) {
            int fv[4], fs = 0;
            for (int k = 0; k < 4; k++) {
                int b[3];
                b[a] = sd; b[ua] = k & 1; b[va] = k >> 1;
                fv[k] = b[0] + 2 * b[1] + 4 * b[2];
                fs |= ((sg >> fv[k]) & 1) << k;
            }
            if (fs != 6 && fs != 9) continue;   // only a diagonal pattern has a saddle decision
            double hf[4] = {g[fv[0]], g[fv[1]], g[fv[2]], g[fv[3]]};
            double den = hf[0] - hf[1] - hf[2] + hf[3];
            double hs = (hf[0] * hf[3] - hf[1] * hf[2]) / den;
            double eb = 0;
            for (int k = 0; k < 4; k++) eb += e[fv[k]];
            // h_s = (h0 h3 - h1 h2) / den: each value enters with weight <= 2 max|h| / |den|
            double amp = 2.0 * (fabs(hf[0]) + fabs(hf[1]) + fabs(hf[2]) + fabs(hf[3])) / fabs(den);
            if (fabs(hs - c) <= 4.0 * amp * eb) {
                for (int k = 0; k < 4; k++) m |= 1u << fv[k];
                r_face = true;
            }
        }
        // fold roots of axis a: A = lower face - c, B = upper - lower
        // (bilinear in the face coordinates u, v); a root solves A = B = 0
        float lo4[4], up4[4], elo[4], eup[4];
        int ilo4[4], iup4[4], nlo = 0, nup = 0;
        for (int k = 0; k < 4; k++) {
            int b[3];
            b[a] = 0; b[ua] = k & 1; b[va] = k >> 1;
            ilo4[k] = b[0] + 2 * b[1] + 4 * b[2];
            b[a] = 1;
            iup4[k] = b[0] + 2 * b[1] + 4 * b[2];
            lo4[k] = gc[ilo4[k]]; elo[k] = e[ilo4[k]];
            up4[k] = gc[iup4[k]]; eup[k] = e[iup4[k]];
            nlo += (sg >> ilo4[k]) & 1;
            nup += (sg >> iup4[k]) & 1;
        }
        if (nlo == 0 || nlo == 4 || nup == 0 || nup == 4) continue;
        const float p0 = lo4[0], p1 = lo4[1] - lo4[0], p2 = lo4[2] - lo4[0], p3 = lo4[3] - lo4[1] - lo4[2] + lo4[0];
        const float d0 = up4[0] - lo4[0], d1 = up4[1] - lo4[1], d2 = up4[2] - lo4[2], d3 = up4[3] - lo4[3];
        const float q0 = d0, q1 = d1 - d0, q2 = d2 - d0, q3 = d3 - d1 - d2 + d0;
        if (q0 == 0.f && q1 == 0.f && q2 == 0.f && q3 == 0.f) continue;
        // (p0 + p1 u)(q2 + q3 u) - (p2 + p3 u)(q0 + q1 u) = 0
        const float A2 = p1 * q3 - p3 * q1, A1 = p0 * q3 + p1 * q2 - p2 * q1 - p3 * q0, A0 = p0 * q2 - p2 * q0;
        const float slack = 2e-3f;
        float us[2];
        int nu = 0;
        const float scale = A1 * A1 + 4.f * fabsf(A2 * A0);
        if (A2 == 0.f) {
            if (A1 != 0.f) us[nu++] = -A0 / A1;
        } else {
            const float disc = A1 * A1 - 4.f * A2 * A0;
            if (fabsf(disc) <= 1e-4f * scale) {
                // a double root within FP32 noise: two roots may merge or part
                const float u2 = -A1 / (2.f * A2);
                if (u2 > -0.01f && u2 < 1.01f) { all = true; break; }
            } else if (disc > 0.f) {
                const float sq = sqrtf(disc), w = A1 >= 0.f ? -0.5f * (A1 + sq) : -0.5f * (A1 - sq);
                if (w != 0.f) { us[nu++] = w / A2; us[nu++] = A0 / w; }
            }
        }
        for (int r = 0; r < nu && !all; r++) {
            const float u = us[r];
            if (!(u > -slack && u < 1.f + slack)) continue;
            const float denB = q2 + q3 * u, denA = p2 + p3 * u;
            const bool useB = fabsf(denB) >= fabsf(denA);
            const float den = useB ? denB : denA;
            if (den == 0.f) { all = true; break; }
            const float v = useB ? -(q0 + q1 * u) / denB : -(p0 + p1 * u) / denA;
            if (!(v > -slack && v < 1.f + slack)) continue;
            // corner errors move A and B at the root by the bilinear weights
            // times the errors, and the root by J^-1 of that
            const float w4[4] = {(1 - u) * (1 - v), u * (1 - v), (1 - u) * v, u * v};
            const float J11 = p1 + p3 * v, J12 = p2 + p3 * u, J21 = q1 + q3 * v, J22 = q2 + q3 * u;
            const float det = fabsf(J11 * J22 - J12 * J21);
            if (!(det > 0.f)) { all = true; break; }
            float share[8], tot = 0.f, bu = 0.f, bv = 0.f;
            for (int q = 0; q < 4; q++) {
                const float slo = infl * fabsf(w4[q]) * elo[q], sup = infl * fabsf(w4[q]) * eup[q];
                const float dul = (fabsf(J22) + fabsf(J12)) * slo / det, dvl = (fabsf(J21) + fabsf(J11)) * slo / det;
                const float duu = fabsf(J12) * sup / det, dvu = fabsf(J11) * sup / det;
                share[ilo4[q]] = dul + dvl;
                share[iup4[q]] = duu + dvu;
                bu += dul + duu;
                bv += dvl + dvu;
            }
            for (int q = 0; q < 8; q++) tot += share[q];
            // a root near the face square's boundary may cross it
            if (fminf(fabsf(u), fabsf(1.f - u)) <= 4.f * bu + 1e-5f || fminf(fabsf(v), fabsf(1.f - v)) <= 4.f * bv + 1e-5f) {
                all = true;
                break;
            }
            if (h * tot > tolf) {
                // re-evaluate the largest contributors until the rest is within tol
                unsigned done = 0;
                float rest = tot;
                for (int it = 0; it < 8 && h * rest > tolf; it++) {
                    int best = -1;
                    for (int q = 0; q < 8; q++)
                        if (!((done >> q) & 1) && (best < 0 || share[q] > share[best])) best = q;
                    done |= 1u << best;
                    rest -= share[best];
                }
                m |= done;
                r_fold = true;
            }
        }
    }
    if (all) m = 0xFF;
    for (int v = 0; v < 8; v++)
        if ((m >> v) & 1) mark[vid[v]] = 1;
    const unsigned act = __activemask();
    const int leader = __ffs(act) - 1, lane = (int)(threadIdx.x & 31);
    if (why) {
        // cubes marked through an edge point, a face saddle, a fold root, and
        // of those all eight corners (one atomic per warp and counter)
        const unsigned b0 = __ballot_sync(act, r_edge), b1 = __ballot_sync(act, r_face),
                       b2 = __ballot_sync(act, all || r_fold), b3 = __ballot_sync(act, all);
        if (lane == leader) {
            if (b0) atomicAdd(&why[0], (unsigned long long)__popc(b0));
            if (b1) atomicAdd(&why[1], (unsigned long long)__popc(b1));
            if (b2) atomicAdd(&why[2], (unsigned long long)__popc(b2));
            if (b3) atomicAdd(&why[3], (unsigned long long)__popc(b3));
        }
    }
    if (out_list) {
        const unsigned b = __ballot_sync(act, m != 0);
        unsigned long long base = 0;
        if (lane == leader && b) base = atomicAdd(n_out, (unsigned long long)__popc(b));
        base = __shfl_sync(act, base, leader);
        if (m != 0) out_list[base + __popc(b & ((1u << lane) - 1u))] = ci;
    }
}

int gs_tri_marks(const TriCtx &X, const float *d_err, double tol_A, int64_t *d_mark, unsigned long long *d_why,
                 const int64_t *d_in_list, int64_t n_in, int64_t *d_out_list, int64_t *n_out, cudaStream_t st)
{
    if (n_out) *n_out = 0;
    // all cubes: those with a surface only, grouped by corner sign pattern
    // (fewer divergent branches per warp)
    int32_t *order = nullptr;
    int64_t nt = d_in_list ? n_in : X.ncubes;
    if (!d_in_list) {
        int rc = tri_order(X, &order, &nt, st);
        if (rc) return rc;
    }
    if (nt <= 0) {
        gs_free(order, st);
        return GS_OK;
    }
    unsigned long long *d_n = nullptr;
    if (d_out_list) {
        int rc = gs_alloc((void **)&d_n, sizeof(unsigned long long), st);
        if (rc) { gs_free(order, st); return rc; }
        GS_CHECK(cudaMemsetAsync(d_n, 0, sizeof(unsigned long long), st));
    }
    GS_LAUNCH(k_tri_marks, (unsigned)((nt + 127) / 128), 128, 0, st)(X, d_err, tol_A, d_mark, d_why, d_in_list, order,
                                                                    nt, d_out_list, d_n);
    gs_free(order, st);
    GS_CHECK(cudaGetLastError());
    if (d_out_list) {
        unsigned long long h = 0;
        cudaError_t e = cudaMemcpyAsync(&h, d_n, sizeof(h), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = gs_sync(st);
        gs_free(d_n, st);
        if (e != cudaSuccess) return gs_fail_cuda(e, "marked cube count", __FILE__, __LINE__);
        if (n_out) *n_out = (int64_t)h;
    }
    return GS_OK;
}

// ---------------------------------------------------------------- adjoint
// With the cube set and the topology held fixed, every mesh vertex is a
// function of the lattice values of one cube: an edge point of its edge's
// two end values (eq intersection), an extreme point of its owner cube's
// eight corners through the fold equations A = B = 0 (eq fold1), a critical
// point of the two fold roots that define it.  k_vertex_adjoint pulls
// dL/dp back to dL/dphi at the lattice vertices (lambda).

// derivatives of a fold root (u, v) of axis a with respect to the eight
// corner values: J (du, dv) = -(dA, dB), with A the bilinear interpolant of
// the lower face minus c and B that of upper minus lower, J their Jacobian
__device__ void fold_root_grad(const double *g, int a, double u, double v, double du[8], double dv[8])
{
    int ua, va;
    axes_other(a, ua, va);
    double lo[4], up[4];
    int ilo[4], iup[4];
    for (int k = 0; k < 4; k++) {
        int b[3];
        b[a] = 0; b[ua] = k & 1; b[va] = k >> 1;
        ilo[k] = b[0] + 2 * b[1] + 4 * b[2];
        b[a] = 1;
        iup[k] = b[0] + 2 * b[1] + 4 * b[2];
        lo[k] = g[ilo[k]];
        up[k] = g[iup[k]];
    }
    double p1 = lo[1] - lo[0], p2 = lo[2] - lo[0], p3 = lo[3] - lo[1] - lo[2] + lo[0];
    double d0 = up[0] - lo[0], d1 = up[1] - lo[1], d2 = up[2] - lo[2], d3 = up[3] - lo[3];
    double q1 = d1 - d0, q2 = d2 - d0, q3 = d3 - d1 - d2 + d0;
    double J11 = p1 + p3 * v, J12 = p2 + p3 * u, J21 = q1 + q3 * v, J22 = q2 + q3 * u;
    double det = J11 * J22 - J12 * J21;
    double inv = det != 0.0 ? 1.0 / det : 0.0;
    double w[4] = {(1 - u) * (1 - v), u * (1 - v), (1 - u) * v, u * v};
    for (int k = 0; k < 8; k++) { du[k] = 0; dv[k] = 0; }
    for (int k = 0; k < 4; k++) {
        // lower corner: dA = w, dB = -w; upper corner: dA = 0, dB = w
        du[ilo[k]] = -w[k] * (J22 + J12) * inv;
        dv[ilo[k]] = w[k] * (J21 + J11) * inv;
        du[iup[k]] = J12 * w[k] * inv;
        dv[iup[k]] = -J11 * w[k] * inv;
    }
}

struct AdjCtx {
    TriCtx X;
    GsHash lat;                 // lattice vertex key -> id
    GsHash cub;                 // cube key -> index
    const uint64_t *mkeys;      // mesh vertex keys
    const double *gv;           // dL/dp per mesh vertex [n, 3]
    int64_t nm;
    double *lambda;             // dL/dphi per lattice vertex
};

__device__ __forceinline__ int64_t adj_lat(const AdjCtx &C, int64_t x, int64_t y, int64_t z)
{
    int64_t s = gs_hash_find(C.lat, gk_make(x, y, z, GT_VERT, 0));
    return s < 0 ? -1 : (int64_t)C.lat.vals[s];
}

__global__ void __launch_bounds__(128) k_vertex_adjoint(AdjCtx C, unsigned *status)
{
    int64_t m = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (m >= C.nm) return;
    const double G[3] = {C.gv[3 * m], C.gv[3 * m + 1], C.gv[3 * m + 2]};
    if (G[0] == 0.0 && G[1] == 0.0 && G[2] == 0.0) return;
    const uint64_t K = C.mkeys[m];
    const unsigned type = gk_type(K), lvl = gk_level(K);
    const int64_t L[3] = {gk_x(K), gk_y(K), gk_z(K)};
    const int64_t sc = (int64_t)1 << (C.X.max_depth - (int)lvl);
    const double h = ldexp(C.X.min_edge, C.X.max_depth - (int)lvl);
    const double c = C.X.c;
    if (type <= 2) {
        // edge point: t = (c - g0) / (g1 - g0) along axis a
        const int a = (int)type;
        int64_t L1[3] = {L[0], L[1], L[2]};
        L1[a] += sc;
        int64_t i0 = adj_lat(C, L[0], L[1], L[2]), i1 = adj_lat(C, L1[0], L1[1], L1[2]);
        if (i0 < 0 || i1 < 0) { atomicOr(status, GS_ST_LOOKUP); return; }
        double g0 = C.X.phi[i0], g1 = C.X.phi[i1], dg = g1 - g0;
        if (dg == 0.0) return;
        double t = (c - g0) / dg;
        atomicAdd(&C.lambda[i0], G[a] * h * (-(1.0 - t) / dg));
        atomicAdd(&C.lambda[i1], G[a] * h * (-t / dg));
        return;
    }
    // extreme (8 + 4a + 2 side + rank) or critical (20 + 4 (a + b - 1) + 2 i + j) point
    int64_t cube[3] = {L[0], L[1], L[2]};
    int fa = -1, fr = 0, fb = -1, fj = 0;
    if (type >= 8 && type < 20) {
        const int code = (int)type - 8;
        fa = code >> 2;
        fr = code & 1;
        if (!((code >> 1) & 1)) cube[fa] -= sc;   // the end on the owner's upper face
    } else if (type >= 20 && type < 32) {
        const int code = (int)type - 20, pr = code >> 2;
        fa = pr == 2 ? 1 : 0;
        fb = pr == 0 ? 1 : 2;
        fr = (code >> 1) & 1;
        fj = code & 1;
    } else {
        return;
    }
    int64_t s = gs_hash_find(C.cub, gk_make(cube[0] / sc, cube[1] / sc, cube[2] / sc, GT_CUBE, lvl));
    if (s < 0) { atomicOr(status, GS_ST_LOOKUP); return; }
    const int64_t ci = (int64_t)C.cub.vals[s];
    double g[8];
    int64_t vid[8];
    for (int v = 0; v < 8; v++) {
        vid[v] = C.X.cvid[ci * 8 + v];
        g[v] = C.X.phi[vid[v]];
    }
    double dp[3][8];
    for (int q = 0; q < 3; q++)
        for (int v = 0; v < 8; v++) dp[q][v] = 0.0;
    double ru[2], rv[2], du[8], dv[8];
    int ua, va;
    int nr = fold_solve(g, fa, c, ru, rv);
    if (fr >= nr) { atomicOr(status, GS_ST_LOOKUP); return; }
    axes_other(fa, ua, va);
    fold_root_grad(g, fa, ru[fr], rv[fr], du, dv);
    if (fb < 0) {
        for (int v = 0; v < 8; v++) { dp[ua][v] = du[v]; dp[va][v] = dv[v]; }
    } else {
        // coordinate fa from the b-root, the other two from the a-root (the
        // shared coordinate is the a-root's)
        const int cc = 3 - fa - fb;
        for (int v = 0; v < 8; v++) {
            dp[fb][v] = fb == ua ? du[v] : dv[v];
            dp[cc][v] = cc == ua ? du[v] : dv[v];
        }
        int ub, vb;
        axes_other(fb, ub, vb);
        int nb = fold_solve(g, fb, c, ru, rv);
        if (fj >= nb) { atomicOr(status, GS_ST_LOOKUP); return; }
        fold_root_grad(g, fb, ru[fj], rv[fj], du, dv);
        for (int v = 0; v < 8; v++) dp[fa][v] = fa == ub ? du[v] : dv[v];
    }
    for (int v = 0; v < 8; v++) {
        double lam = h * (G[0] * dp[0][v] + G[1] * dp[1][v] + G[2] * dp[2][v]);
        if (lam != 0.0) atomicAdd(&C.lambda[vid[v]], lam);
    }
}

// volume sum p0.(p1 x p2)/6 and area sum |(p1-p0) x (p2-p0)|/2 of a closed,
// outward-oriented mesh, with their gradients per vertex (nullable)
__global__ void __launch_bounds__(256) k_volume_area(const double *__restrict__ v, const int32_t *__restrict__ tri,
                                                     int64_t nt, double *acc, double *gV, double *gA)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    double vol = 0.0, area = 0.0;
    if (t < nt) {
        const int32_t i[3] = {tri[3 * t], tri[3 * t + 1], tri[3 * t + 2]};
        double p[3][3];
        for (int k = 0; k < 3; k++)
            for (int q = 0; q < 3; q++) p[k][q] = v[3 * (int64_t)i[k] + q];
        auto cross = [](const double *x, const double *y, double *o) {
            o[0] = x[1] * y[2] - x[2] * y[1];
            o[1] = x[2] * y[0] - x[0] * y[2];
            o[2] = x[0] * y[1] - x[1] * y[0];
        };
        double c12[3], c20[3], c01[3];
        cross(p[1], p[2], c12);
        cross(p[2], p[0], c20);
        cross(p[0], p[1], c01);
        vol = (p[0][0] * c12[0] + p[0][1] * c12[1] + p[0][2] * c12[2]) / 6.0;
        double e1[3], e2[3], n[3];
        for (int q = 0; q < 3; q++) { e1[q] = p[1][q] - p[0][q]; e2[q] = p[2][q] - p[0][q]; }
        cross(e1, e2, n);
        double nn = sqrt(n[0] * n[0] + n[1] * n[1] + n[2] * n[2]);
        area = 0.5 * nn;
        if (gV)
            for (int q = 0; q < 3; q++) {
                atomicAdd(&gV[3 * (int64_t)i[0] + q], c12[q] / 6.0);
                atomicAdd(&gV[3 * (int64_t)i[1] + q], c20[q] / 6.0);
                atomicAdd(&gV[3 * (int64_t)i[2] + q], c01[q] / 6.0);
            }
        if (gA && nn > 0.0) {
            double nh[3] = {n[0] / nn, n[1] / nn, n[2] / nn};
            // d area / d p_k = n_hat x (p_{k+2} - p_{k+1}) / 2
            for (int k = 0; k < 3; k++) {
                double d[3], o[3];
                for (int q = 0; q < 3; q++) d[q] = p[(k + 2) % 3][q] - p[(k + 1) % 3][q];
                cross(nh, d, o);
                for (int q = 0; q < 3; q++) atomicAdd(&gA[3 * (int64_t)i[k] + q], 0.5 * o[q]);
            }
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        vol += __shfl_xor_sync(0xffffffffu, vol, o);
        area += __shfl_xor_sync(0xffffffffu, area, o);
    }
    if ((threadIdx.x & 31) == 0) {
        atomicAdd(&acc[0], vol);
        atomicAdd(&acc[1], area);
    }
}

int gs_vertex_adjoint(const TriCtx &X, const uint64_t *d_lat_keys, int64_t nlat, const uint64_t *d_mkeys,
                      const double *d_gv, int64_t nm, double *d_lambda, unsigned *d_status, cudaStream_t st)
{
    AdjCtx C;
    C.X = X;
    C.mkeys = d_mkeys;
    C.gv = d_gv;
    C.nm = nm;
    C.lambda = d_lambda;
    int rc = gs_hash_make(&C.lat, nlat, st);
    if (rc) return rc;
    rc = gs_hash_make(&C.cub, X.ncubes, st);
    if (rc) { gs_hash_free(&C.lat, st); return rc; }
    GS_CHECK(cudaMemsetAsync(d_lambda, 0, sizeof(double) * (size_t)(nlat + 1), st));
    if (nlat > 0) GS_LAUNCH(k_hash_index, (unsigned)((nlat + 255) / 256), 256, 0, st)(C.lat, d_lat_keys, nlat, d_status);
    if (X.ncubes > 0)
        GS_LAUNCH(k_hash_index, (unsigned)((X.ncubes + 255) / 256), 256, 0, st)(C.cub, X.cubes, X.ncubes, d_status);
    if (nm > 0) GS_LAUNCH(k_vertex_adjoint, (unsigned)((nm + 127) / 128), 128, 0, st)(C, d_status);
    gs_hash_free(&C.lat, st);
    gs_hash_free(&C.cub, st);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

int gs_volume_area_dev(const double *d_v, const int32_t *d_tri, int64_t nt, double *d_acc, double *d_gV, double *d_gA,
                       cudaStream_t st)
{
    GS_CHECK(cudaMemsetAsync(d_acc, 0, 2 * sizeof(double), st));
    if (nt > 0)
        GS_LAUNCH(k_volume_area, (unsigned)((nt + 255) / 256), 256, 0, st)(d_v, d_tri, nt, d_acc, d_gV, d_gA);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}
