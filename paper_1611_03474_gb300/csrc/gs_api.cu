// gs_api.cu -- host orchestration and the C ABI (include/gsmesh.h).
//
// mesh_gaussian_surface runs, on one stream:
//   upload -> atom prep (cutoff radii, bounding box) -> root grid (host)
//   -> cell list -> for each level: tensor accumulation, estimation,
//   compaction -> conformity -> lattice vertices and their field values ->
//   face neighbours -> triangulation (count, scan, emit) -> weld -> download.
// The host waits once per level for the next level's size.
#include <cmath>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <mutex>
#include <vector>

#include "gs_host.cuh"

#include <nvtx3/nvToolsExt.h>

#include <algorithm>
#include <initializer_list>
#include <memory>
#include <atomic>
#include <condition_variable>
#include <string>
#include <thread>
#include <vector>

extern "C" gs_options gs_default_options(void)
{
    gs_options o;
    memset(&o, 0, sizeof(o));
    o.min_edge = 0.25;
    o.precision_mode = GS_PREC_FP64;
    o.cutoff_rel = 1e-8;
    return o;
}

extern "C" const char *gs_status_string(int s)
{
    switch (s) {
    case GS_OK: return "ok";
    case GS_ERR_ARG: return "invalid argument";
    case GS_ERR_OOM: return "out of memory";
    case GS_ERR_CAPACITY: return "internal capacity exceeded";
    case GS_ERR_TIMEOUT: return "timeout";
    case GS_ERR_CUDA: return "CUDA error";
    case GS_ERR_DEVICE_STATUS: return "device status error";
    default: return "unknown status";
    }
}

extern "C" int gs_memory_kind(const void *p) { return gs_host_kind(p); }

extern "C" int64_t gs_struct_size(int which)
{
    switch (which) {
    case 0: return (int64_t)sizeof(gs_stats);
    case 1: return (int64_t)sizeof(gs_options);
    case 2: return (int64_t)sizeof(gs_mesh);
    default: return -1;
    }
}

extern "C" void mesh_free(gs_mesh *m)
{
    if (!m) return;
    if (m->on_device) {
        cudaFree(m->vertices); cudaFree(m->triangles); cudaFree(m->vertex_keys); cudaFree(m->cube_keys);
    } else {
        free(m->vertices); free(m->triangles); free(m->vertex_keys); free(m->cube_keys);
    }
    memset(m, 0, sizeof(*m));
}

// device counters of one call (gs_stats fields and internal tallies)
#define GS_NCNT 40

static bool on_device(const void *p)
{
    cudaPointerAttributes a;
    if (cudaPointerGetAttributes(&a, p) != cudaSuccess) { cudaGetLastError(); return false; }
    return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// per-device one-time set-up: quadrature tables, a memory pool that keeps its memory
static std::mutex g_init_mu;
static bool g_dev_ready[64];
static int device_setup(void)
{
    gs_guard_begin();   // every API call starts here: the call's fault-injection state
    int dev = 0;
    GS_CHECK(cudaGetDevice(&dev));
    std::lock_guard<std::mutex> lk(g_init_mu);
    if (dev >= 0 && dev < 64 && g_dev_ready[dev]) return GS_OK;
    int rc = gs_quadrature_init();
    if (!rc) rc = gs_field_init();
    if (rc) return rc;
    cudaMemPool_t pool;
    if (cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
        uint64_t thr = ~0ull;
        cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
    cudaGetLastError();
    if (dev >= 0 && dev < 64) g_dev_ready[dev] = true;
    return GS_OK;
}

// NVTX range for the lifetime of a scope (a phase or a level), visible in
// timeline profilers; a no-op without one attached
struct NvtxRange {
    bool on = true;
    explicit NvtxRange(const char *name) { nvtxRangePushA(name); }
    void end()
    {
        if (on) nvtxRangePop();
        on = false;
    }
    ~NvtxRange() { end(); }
};

// a simple scope guard for stream-ordered device buffers
struct DevBufs {
    cudaStream_t st;
    std::vector<void *> ptrs;
    explicit DevBufs(cudaStream_t s) : st(s) {}
    template <typename T> int get(T **p, size_t count)
    {
        int rc = gs_alloc((void **)p, sizeof(T) * (count ? count : 1), st);
        if (!rc) ptrs.push_back((void *)*p);
        return rc;
    }
    void keep(void *p) { if (p) ptrs.push_back(p); }
    void release(void *p)
    {
        if (!p) return;
        for (auto &q : ptrs)
            if (q == p) { gs_free(q, st); q = nullptr; }
    }
    // stop tracking p without freeing it (a callee frees or replaces it)
    void forget(void *p)
    {
        if (!p) return;
        for (auto &q : ptrs)
            if (q == p) q = nullptr;
    }
    ~DevBufs()
    {
        for (void *p : ptrs) gs_free(p, st);
    }
};

struct Timer {
    cudaStream_t st;
    std::vector<cudaEvent_t> ev;
    explicit Timer(cudaStream_t s) : st(s) {}
    int mark()
    {
        cudaEvent_t e;
        cudaEventCreate(&e);
        cudaEventRecord(e, st);
        ev.push_back(e);
        return (int)ev.size() - 1;
    }
    double ms(int a, int b)
    {
        float t = 0;
        cudaEventElapsedTime(&t, ev[a], ev[b]);
        return t;
    }
    ~Timer()
    {
        for (auto e : ev) cudaEventDestroy(e);
    }
};

static int check_status(unsigned *d_status, cudaStream_t st, const char *stage)
{
    unsigned h = 0;
    GS_CHECK(cudaMemcpyAsync(&h, d_status, sizeof(unsigned), cudaMemcpyDeviceToHost, st));
    GS_CHECK(gs_sync(st));
    if (h & GS_ST_INPUT) return gs_fail(GS_ERR_ARG, "non-finite or negative atom data");
    if (h & GS_ST_CAPACITY) return gs_fail(GS_ERR_CAPACITY, "%s: internal table full", stage);
    if (h) return gs_fail(GS_ERR_DEVICE_STATUS, "%s: device status 0x%x", stage, h);
    return GS_OK;
}

// root grid of section 2.2: edge h0 = min_edge * 2^max_depth, origin aligned
// to h0, covering the atoms' bounding box grown by the largest cutoff radius
static int root_grid(const double bbox[6], double pad, double min_edge, int max_depth, double origin[3],
                     int64_t nroot[3], double *h0)
{
    *h0 = ldexp(min_edge, max_depth);
    for (int a = 0; a < 3; a++) {
        origin[a] = *h0 * floor((bbox[a] - pad) / *h0);
        int64_t m = (int64_t)ceil((bbox[3 + a] + pad - origin[a]) / *h0);
        nroot[a] = m < 1 ? 1 : m;
        if (((nroot[a] << max_depth) + 1) > (int64_t)GK_MASK)
            return gs_fail(GS_ERR_ARG, "lattice exceeds 2^18 points along an axis");
    }
    return GS_OK;
}

struct Prepared {
    GsProblem P;
    GsAtomsSoA soa;
    int32_t *cell_start;
    int32_t *perm;   // cell-ordered atom -> input index
};

// upload, prep, cell list; buffers registered in B
// The FP32 form keeps every weight exp(D r^2) finite and every factor of a
// term inside the cutoff above the FP32 flush-to-zero range when D R^2 <= 80
// for the largest cutoff radius R (R^2 = r^2 + K/D)
static int check_fp32_range(const GsProblem &P)
{
    if (P.D * P.pad * P.pad > 80.0)
        return gs_fail(GS_ERR_ARG, "D r^2 plus the cutoff exponent exceeds 80: outside the FP32 range of the mixed "
                                   "form; use the FP64 form");
    return GS_OK;
}

static int prepare(const double *atoms, const double *radii, int64_t n, double D, double c, double cutoff_rel,
                   double precision, double min_edge, int max_depth, DevBufs &B, unsigned *d_status, Prepared *out,
                   gs_stats *stats, Timer &T)
{
    cudaStream_t st = B.st;
    const double *d_xyz = atoms, *d_r = radii;
    int t0 = T.mark();
    if (!on_device(atoms)) {
        double *p;
        int rc = B.get(&p, 3 * (size_t)n);
        if (rc) return rc;
        rc = gs_copy_from_host(p, atoms, sizeof(double) * 3 * (size_t)n, st);
        if (rc) return rc;
        d_xyz = p;
    }
    if (!on_device(radii)) {
        double *p;
        int rc = B.get(&p, (size_t)n);
        if (rc) return rc;
        rc = gs_copy_from_host(p, radii, sizeof(double) * (size_t)n, st);
        if (rc) return rc;
        d_r = p;
    }
    int t1 = T.mark();
    double KD = -log(cutoff_rel * c) / D;
    double *d_R2, *d_w;
    int rc = B.get(&d_R2, (size_t)n);
    if (!rc) rc = B.get(&d_w, (size_t)n);
    if (rc) return rc;
    double bbox[6], r2max;
    rc = gs_prep_atoms(d_xyz, d_r, n, D, KD, d_R2, d_w, bbox, &r2max, d_status, st);
    if (rc) return rc;
    rc = check_status(d_status, st, "prep");
    if (rc) return rc;
    GsProblem &P = out->P;
    memset(&P, 0, sizeof(P));
    P.n = n; P.D = D; P.c = c; P.KD = KD; P.precision = precision; P.min_edge = min_edge; P.max_depth = max_depth;
    P.pad = sqrt(r2max);
    double h0;
    rc = root_grid(bbox, P.pad, min_edge, max_depth, P.origin, P.nroot, &h0);
    if (rc) return rc;
    // cell edge: half the cutoff radius balances candidate volume against row count
    P.cell = 0.5 * P.pad;
    if (P.cell <= 0) P.cell = h0;
    P.inv_cell = 1.0 / P.cell;
    P.cell_f = (float)P.cell;
    P.inv_cell_f = (float)P.inv_cell;
    P.pad_f = (float)P.pad;
    {
        // min_edge = k 2^e with k < 64 and indices < 2^18: index * spacing fits 24 bits
        int ex;
        double mant = frexp(min_edge, &ex);
        double k64 = ldexp(mant, 6);
        P.lat_exact_f32 = (k64 == floor(k64)) ? 1 : 0;
    }
    int64_t ncell = 1;
    for (int a = 0; a < 3; a++) {
        double ext = (double)P.nroot[a] * h0;
        int64_t m = (int64_t)ceil(ext / P.cell) + 1;
        if (m > (1 << 20)) return gs_fail(GS_ERR_ARG, "cell grid too large");
        P.cdim[a] = (int)m;
        ncell *= m;
    }
    if (ncell > (int64_t)1 << 31) return gs_fail(GS_ERR_ARG, "cell grid too large");
    int32_t *perm;
    rc = B.get(&out->cell_start, (size_t)ncell + 1);
    if (!rc) rc = B.get(&perm, (size_t)n);
    if (rc) return rc;
    rc = gs_build_cells(d_xyz, n, P.origin, P.cell, P.cdim, out->cell_start, perm, st);
    if (rc) return rc;
    GsAtomsSoA &S = out->soa;
    rc = B.get(&S.x, (size_t)n);
    if (!rc) rc = B.get(&S.y, (size_t)n);
    if (!rc) rc = B.get(&S.z, (size_t)n);
    if (!rc) rc = B.get(&S.r, (size_t)n);
    if (!rc) rc = B.get(&S.R2, (size_t)n);
    if (!rc) rc = B.get(&S.w, (size_t)n);
    if (!rc) rc = B.get(&S.fx, (size_t)n);
    if (!rc) rc = B.get(&S.fy, (size_t)n);
    if (!rc) rc = B.get(&S.fz, (size_t)n);
    if (!rc) rc = B.get(&S.hx, (size_t)n);
    if (!rc) rc = B.get(&S.lx, (size_t)n);
    if (!rc) rc = B.get(&S.hy, (size_t)n);
    if (!rc) rc = B.get(&S.ly, (size_t)n);
    if (!rc) rc = B.get(&S.hz, (size_t)n);
    if (!rc) rc = B.get(&S.lz, (size_t)n);
    if (!rc) rc = B.get(&S.fw, (size_t)n);
    if (!rc) rc = B.get(&S.fR2, (size_t)n);
    if (!rc) rc = B.get(&S.fr2, (size_t)n);
    if (!rc) rc = B.get(&S.lr2, (size_t)n);
    if (rc) return rc;
    out->perm = perm;
    rc = gs_gather_atoms(perm, n, d_xyz, d_r, d_R2, d_w, P.origin, P.cell, P.cdim, &S, st);
    if (rc) return rc;
    P.ax = S.x; P.ay = S.y; P.az = S.z; P.ar = S.r; P.aR2 = S.R2; P.aw = S.w;
    P.fx = S.fx; P.fy = S.fy; P.fz = S.fz;
    P.hx = S.hx; P.lx = S.lx; P.hy = S.hy; P.ly = S.ly; P.hz = S.hz; P.lz = S.lz; P.fw = S.fw; P.fR2 = S.fR2; P.fr2 = S.fr2;
    P.lr2 = S.lr2;
    P.cell_start = out->cell_start;
    int t2 = T.mark();
    if (stats) {
        GS_CHECK(gs_sync(st));
        stats->ms_upload = T.ms(t0, t1);
        stats->ms_bin = T.ms(t1, t2);
    }
    return GS_OK;
}

// the batched form's extra level state: the problem records (device), the
// parents' molecule indices, the root blocks' valid children (level 0),
// and outputs: the accepted cubes' molecule indices (one array per part),
// the next parents' molecule indices and per-molecule decision counts
struct LevelBatch {
    const GsProblem *d_probs = nullptr;
    const int32_t *pmol = nullptr;
    const uint8_t *pvmask = nullptr;
    std::vector<int32_t *> acc_mol;
    int32_t *next_mol = nullptr;
    unsigned long long *molcnt = nullptr;
};

// process one level in chunks of parents; appends accepted keys; returns the next parents
// d_parA (re-expansion only): the parents' tensors [n_oct][64]; *d_nextA
// receives the split cubes' tensors for the next level
static int run_level(const GsProblem &P, int level, const uint64_t *d_parents, int64_t n_oct, int mode,
                     DevBufs &B, std::vector<uint64_t *> &acc_parts, std::vector<int64_t> &acc_counts,
                     uint64_t **d_next, int64_t *n_next, unsigned long long *d_counters, unsigned long long *d_pairs,
                     unsigned long long *d_rechecked, unsigned long long *d_mism, bool both, unsigned *d_status,
                     gs_stats *stats, bool reexpand = false, const double *d_parA = nullptr,
                     double **d_nextA = nullptr, int64_t CH = (int64_t)1 << 21, LevelBatch *lb = nullptr)
{
    cudaStream_t st = B.st;
    // CH: octets per chunk (2^21: 8 GB of FP64 tensors; smaller after an
    // allocation or capacity failure, and 1000 in a debug mode, so that small
    // inputs run the multi-chunk path)
    if (gs_fault_capacity(level)) return gs_fail(GS_ERR_CAPACITY, "level %d: internal table full (injected by GS_FAULT)",
                                                 level);
    std::vector<uint64_t *> nexts;
    std::vector<double *> nextAs;
    std::vector<int32_t *> nextMols;
    std::vector<int64_t> ncnt;
    *d_next = nullptr;
    *n_next = 0;
    if (d_nextA) *d_nextA = nullptr;
    if (lb) lb->next_mol = nullptr;
    // frees the chunks' next-level arrays on an error
    auto drop_nexts = [&]() {
        for (size_t i = 0; i < nexts.size(); i++) { gs_free(nexts[i], st); gs_free(nextAs[i], st); gs_free(nextMols[i], st); }
    };
    for (int64_t o0 = 0; o0 < n_oct; o0 += CH) {
        int64_t m = n_oct - o0 < CH ? n_oct - o0 : CH;
        const uint64_t *par = d_parents + o0;
        const int32_t *pmol = lb ? lb->pmol + o0 : nullptr;
        const uint8_t *pvm = lb && lb->pvmask ? lb->pvmask + o0 : nullptr;
        const GsProblem *probs = lb ? lb->d_probs : nullptr;
        uint8_t *dec = nullptr;
        int rc = gs_alloc((void **)&dec, (size_t)m * 8, st);
        if (rc) { drop_nexts(); return rc; }
        float tacc = 0.f;
        if (mode == GS_PREC_MIXED) {
            rc = gs_level_mixed(P, level, par, m, dec, d_pairs, d_rechecked, d_mism, both, d_status, st,
                                stats ? &tacc : nullptr, d_mism + 1, probs, pmol, pvm);
        }
        double *dA = nullptr;
        if (mode != GS_PREC_MIXED) {
            rc = gs_alloc((void **)&dA, sizeof(double) * 64 * 8 * (size_t)m, st);
            if (rc) { gs_free(dec, st); drop_nexts(); return rc; }
            if (reexpand && d_parA) rc = gs_reexpand(d_parA + 64 * o0, m, dA, st);
            else
                rc = gs_accum_f64(P, level, par, pvm, m, dA, d_pairs, d_status, st, stats ? &tacc : nullptr, probs,
                                  pmol);
            if (!rc) rc = gs_estimate_f64(P, level, dA, m * 8, par, pvm, dec, nullptr, st);
        }
        if (stats) { stats->ms_accum += tacc; stats->n_accum_launches++; }
        if (!rc && lb) rc = gs_level_count_mol(dec, m * 8, pmol, lb->molcnt, st);
        uint64_t *acc = nullptr;
        int32_t *accm = nullptr;
        if (!rc) rc = gs_alloc((void **)&acc, sizeof(uint64_t) * (size_t)m * 8, st);
        if (!rc && lb) rc = gs_alloc((void **)&accm, sizeof(int32_t) * (size_t)m * 8, st);
        uint64_t *nx = nullptr;
        double *nA = nullptr;
        int32_t *nm = nullptr;
        int64_t nn = 0, na = 0;
        if (!rc)
            rc = gs_level_compact(P, level, par, pvm, m, dec, &nx, &nn, acc, m * 8, &na, d_counters, st,
                                  reexpand ? dA : nullptr, reexpand ? &nA : nullptr, pmol, lb ? &nm : nullptr, accm);
        gs_free(dec, st);
        gs_free(dA, st);
        if (rc) {
            gs_free(acc, st); gs_free(accm, st); gs_free(nx, st); gs_free(nA, st); gs_free(nm, st);
            drop_nexts();
            return rc;
        }
        acc_parts.push_back(acc);
        acc_counts.push_back(na);
        if (lb) lb->acc_mol.push_back(accm);
        if (nx) { nexts.push_back(nx); nextAs.push_back(nA); nextMols.push_back(nm); ncnt.push_back(nn); }
    }
    int64_t total = 0;
    for (auto v : ncnt) total += v;
    if (nexts.size() == 1) {
        *d_next = nexts[0];
        if (d_nextA) *d_nextA = nextAs[0];
        else gs_free(nextAs[0], st);
        if (lb) lb->next_mol = nextMols[0];
    } else if (total > 0) {
        int rc = gs_alloc((void **)d_next, sizeof(uint64_t) * (size_t)total, st);
        if (!rc && reexpand && d_nextA) rc = gs_alloc((void **)d_nextA, sizeof(double) * 64 * (size_t)total, st);
        if (!rc && lb) rc = gs_alloc((void **)&lb->next_mol, sizeof(int32_t) * (size_t)total, st);
        if (rc) { drop_nexts(); return rc; }
        int64_t off = 0;
        for (size_t i = 0; i < nexts.size(); i++) {
            GS_CHECK(cudaMemcpyAsync(*d_next + off, nexts[i], sizeof(uint64_t) * (size_t)ncnt[i],
                                     cudaMemcpyDeviceToDevice, st));
            if (reexpand && d_nextA && nextAs[i])
                GS_CHECK(cudaMemcpyAsync(*d_nextA + 64 * off, nextAs[i], sizeof(double) * 64 * (size_t)ncnt[i],
                                         cudaMemcpyDeviceToDevice, st));
            if (lb)
                GS_CHECK(cudaMemcpyAsync(lb->next_mol + off, nextMols[i], sizeof(int32_t) * (size_t)ncnt[i],
                                         cudaMemcpyDeviceToDevice, st));
            off += ncnt[i];
            gs_free(nexts[i], st);
            gs_free(nextAs[i], st);
            gs_free(nextMols[i], st);
        }
    }
    *n_next = total;
    return GS_OK;
}

struct MeshDev {
    double *vxyz = nullptr;
    uint64_t *vkeys = nullptr;
    int32_t *tri = nullptr;
    uint64_t *cubes = nullptr;
    int64_t nv = 0, nt = 0, nc = 0;
};

static int finish_output(MeshDev &M, const gs_options &o, gs_mesh *out, cudaStream_t st)
{
    out->n_vertices = M.nv;
    out->n_triangles = M.nt;
    out->n_cubes = M.nc;
    if (o.device_output) {
        // hand over as plain cudaMalloc memory (mesh_free uses cudaFree)
        out->on_device = 1;
        double *v = nullptr; int32_t *t = nullptr; uint64_t *k = nullptr, *cb = nullptr;
        GS_CHECK(cudaMalloc(&v, sizeof(double) * 3 * (size_t)(M.nv + 1)));
        GS_CHECK(cudaMalloc(&t, sizeof(int32_t) * 3 * (size_t)(M.nt + 1)));
        GS_CHECK(cudaMalloc(&k, sizeof(uint64_t) * (size_t)(M.nv + 1)));
        GS_CHECK(cudaMalloc(&cb, sizeof(uint64_t) * (size_t)(M.nc + 1)));
        out->vertices = v; out->triangles = t; out->vertex_keys = k; out->cube_keys = cb;
        if (M.nv) {
            GS_CHECK(cudaMemcpyAsync(v, M.vxyz, sizeof(double) * 3 * (size_t)M.nv, cudaMemcpyDeviceToDevice, st));
            GS_CHECK(cudaMemcpyAsync(k, M.vkeys, sizeof(uint64_t) * (size_t)M.nv, cudaMemcpyDeviceToDevice, st));
        }
        if (M.nt) GS_CHECK(cudaMemcpyAsync(t, M.tri, sizeof(int32_t) * 3 * (size_t)M.nt, cudaMemcpyDeviceToDevice, st));
        if (M.nc) GS_CHECK(cudaMemcpyAsync(cb, M.cubes, sizeof(uint64_t) * (size_t)M.nc, cudaMemcpyDeviceToDevice, st));
    } else {
        out->on_device = 0;
        out->vertices = (double *)malloc(sizeof(double) * 3 * (size_t)(M.nv + 1));
        out->triangles = (int32_t *)malloc(sizeof(int32_t) * 3 * (size_t)(M.nt + 1));
        out->vertex_keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(M.nv + 1));
        out->cube_keys = (uint64_t *)malloc(sizeof(uint64_t) * (size_t)(M.nc + 1));
        if (!out->vertices || !out->triangles || !out->vertex_keys || !out->cube_keys)
            return gs_fail(GS_ERR_OOM, "host output allocation");
        if (M.nv) {
            GS_CHECK(cudaMemcpyAsync(out->vertices, M.vxyz, sizeof(double) * 3 * (size_t)M.nv, cudaMemcpyDeviceToHost, st));
            GS_CHECK(cudaMemcpyAsync(out->vertex_keys, M.vkeys, sizeof(uint64_t) * (size_t)M.nv, cudaMemcpyDeviceToHost, st));
        }
        if (M.nt)
            GS_CHECK(cudaMemcpyAsync(out->triangles, M.tri, sizeof(int32_t) * 3 * (size_t)M.nt, cudaMemcpyDeviceToHost, st));
        if (M.nc)
            GS_CHECK(cudaMemcpyAsync(out->cube_keys, M.cubes, sizeof(uint64_t) * (size_t)M.nc, cudaMemcpyDeviceToHost, st));
    }
    GS_CHECK(gs_sync(st));
    return GS_OK;
}

// the mesh into caller-owned buffers (cudaMemcpyDefault: host or device)
static int finish_into(MeshDev &M, gs_mesh_buffers *b, cudaStream_t st)
{
    b->n_vertices = M.nv;
    b->n_triangles = M.nt;
    b->n_cubes = M.nc;
    if (M.nv > b->cap_vertices || M.nt > b->cap_triangles || (b->cube_keys && M.nc > b->cap_cubes))
        return gs_fail(GS_ERR_CAPACITY, "output buffers too small: the mesh has %lld vertices, %lld triangles, %lld cubes",
                       (long long)M.nv, (long long)M.nt, (long long)M.nc);
    int rc = GS_OK;
    if (M.nv) {
        rc = gs_copy_to_host(b->vertices, M.vxyz, sizeof(double) * 3 * (size_t)M.nv, st);
        if (!rc && b->vertex_keys) rc = gs_copy_to_host(b->vertex_keys, M.vkeys, sizeof(uint64_t) * (size_t)M.nv, st);
    }
    if (!rc && M.nt) rc = gs_copy_to_host(b->triangles, M.tri, sizeof(int32_t) * 3 * (size_t)M.nt, st);
    if (!rc && M.nc && b->cube_keys) rc = gs_copy_to_host(b->cube_keys, M.cubes, sizeof(uint64_t) * (size_t)M.nc, st);
    if (rc) return rc;
    GS_CHECK(gs_sync(st));
    return GS_OK;
}

// triangulate the final cubes given lattice vertex values; shared by the
// molecule path and the grid entry point
// cubes of different sizes in the final set (constrained vertex values)
struct MixInfo {
    const uint8_t *mixed;       // per cube, or null when no cube has a neighbour of another size
    GsHash hc, hv;              // cube key -> index; lattice-vertex key -> slot
    const uint64_t *vslot_id;   // slot -> lattice vertex id
};

static int surface_from_values(const GsProblem &P, const uint64_t *d_cubes, int64_t nc, const int32_t *d_cvid,
                               const double *d_phi, DevBufs &B, unsigned *d_status, unsigned long long *d_tcount,
                               MeshDev &M, gs_stats *stats, Timer &T, const MixInfo *mx = nullptr)
{
    cudaStream_t st = B.st;
    int t0 = T.mark();
    int32_t *nbr = nullptr;
    int rc = gs_neighbours(d_cubes, nc, &nbr, d_status, st);
    if (rc) return rc;
    B.keep(nbr);
    TriCtx X;
    if (mx && mx->mixed) {
        X.mixed = mx->mixed; X.hc = mx->hc; X.hv = mx->hv; X.vslot_id = mx->vslot_id;
    }
    X.cubes = d_cubes; X.cvid = d_cvid; X.nbr = nbr; X.phi = d_phi; X.ncubes = nc; X.c = P.c;
    for (int a = 0; a < 3; a++) X.origin[a] = P.origin[a];
    X.min_edge = P.min_edge; X.max_depth = P.max_depth;
    uint64_t *tk = nullptr, *pk = nullptr;
    double *pxyz = nullptr;
    int64_t ntri = 0, npt = 0;
    rc = gs_triangulate(X, &tk, &ntri, &pk, &pxyz, &npt, d_tcount, st);
    B.keep(tk); B.keep(pk); B.keep(pxyz);
    if (rc) return rc;
    int t1 = T.mark();
    rc = gs_weld(pk, pxyz, npt, tk, ntri, &M.vkeys, &M.vxyz, &M.nv, &M.tri, d_status, st);
    B.keep(M.vkeys); B.keep(M.vxyz); B.keep(M.tri);
    if (rc) return rc;
    M.nt = ntri;
    int t2 = T.mark();
    rc = check_status(d_status, st, "triangulation");
    if (rc) return rc;
    if (stats) {
        stats->ms_triangulate = T.ms(t0, t1);
        stats->ms_weld = T.ms(t1, t2);
        stats->n_points = npt;
        unsigned long long h[3];
        GS_CHECK(cudaMemcpy(h, d_tcount, sizeof(h), cudaMemcpyDeviceToHost));
        stats->loop_errors = (int64_t)h[0];
        stats->degenerate_ears = (int64_t)h[1];
        stats->n_cubes_surface = (int64_t)h[2];
    }
    return GS_OK;
}

__global__ void k_fill_grid_phi(const uint64_t *vkeys, int64_t nv, const double *vals, int64_t nx, int64_t ny,
                                double *phi)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nv) return;
    uint64_t k = vkeys[i];
    phi[i] = vals[gk_x(k) + (nx + 1) * (gk_y(k) + (ny + 1) * gk_z(k))];
}

__global__ void k_grid_cubes(int64_t nx, int64_t ny, int64_t nz, uint64_t *cubes)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nx * ny * nz) return;
    cubes[i] = gk_make(i % nx, (i / nx) % ny, i / (nx * ny), GT_CUBE, 0);
}

// the level loop of one molecule (section 2.2, steps 1-3): the accepted
// cubes, level by level, in *cubes (device, the caller owns them)
static int single_levels(const GsProblem &P, const gs_options &o, int max_depth, DevBufs &B, Timer &T,
                         unsigned long long *d_cnt, unsigned *d_status, gs_stats *stats, int64_t chunk,
                         bool *retryable, uint64_t **cubes_out, int64_t *nc_out)
{
    cudaStream_t st = B.st;
    int rc = GS_OK;
    std::vector<uint64_t *> acc_all;
    std::vector<int64_t> acc_cnt;
    uint64_t *parents = nullptr;
    double *parentA = nullptr;   // re-expansion: the parents' tensors
    const bool reexpand = o.child_mode == GS_CHILD_REEXPAND;
    int64_t n_oct = 0;
    rc = gs_root_blocks(P, &parents, &n_oct, st);
    if (rc) return rc;
    B.keep(parents);
    for (int l = 0; l <= max_depth && n_oct > 0; l++) {
        char lname[32];
        snprintf(lname, sizeof(lname), "gs: level %d", l);
        NvtxRange nr(lname);
        int ta = T.mark();
        GS_CHECK(cudaMemsetAsync(d_cnt, 0, 5 * sizeof(unsigned long long), st));
        uint64_t *next = nullptr;
        int64_t nn = 0;
        std::vector<uint64_t *> parts;
        std::vector<int64_t> cnts;
        double *nextA = nullptr;
        rc = run_level(P, l, parents, n_oct, o.precision_mode, B, parts, cnts, &next, &nn, d_cnt, d_cnt + 8,
                       d_cnt + 13, d_cnt + 14, (o.debug_flags & 1) != 0, d_status, stats, reexpand, parentA,
                       reexpand ? &nextA : nullptr, (o.debug_flags & 2) ? (int64_t)1000 : chunk);
        if (parentA) B.release(parentA);
        parentA = nextA;
        if (parentA) B.keep(parentA);
        for (size_t i = 0; i < parts.size(); i++) { B.keep(parts[i]); acc_all.push_back(parts[i]); acc_cnt.push_back(cnts[i]); }
        if (parents) B.release(parents);
        if (rc) {
            // out of device memory or of an internal table in the level loop:
            // the caller may try again with smaller level chunks
            if (retryable && (rc == GS_ERR_OOM || rc == GS_ERR_CAPACITY)) *retryable = true;
            gs_free(next, st);
            return rc;
        }
        parents = next;
        B.keep(parents);
        n_oct = nn;
        int tb = T.mark();
        unsigned long long h[5];
        GS_CHECK(cudaMemcpyAsync(h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
        GS_CHECK(gs_sync(st));
        stats->examined[l] = (int64_t)h[0]; stats->discarded[l] = (int64_t)h[1]; stats->accepted[l] = (int64_t)h[2];
        stats->forced[l] = (int64_t)h[3]; stats->split[l] = (int64_t)h[4];
        stats->ms_level[l] = T.ms(ta, tb);
    }
    if (parents) B.release(parents);
    if (parentA) B.release(parentA);
    rc = check_status(d_status, st, "levels");
    if (rc) return rc;
    int64_t nc = 0;
    for (auto v : acc_cnt) nc += v;
    uint64_t *cubes = nullptr;
    rc = gs_alloc((void **)&cubes, sizeof(uint64_t) * (size_t)(nc + 1), st);
    if (rc) return rc;
    {
        int64_t off = 0;
        for (size_t i = 0; i < acc_all.size(); i++) {
            if (acc_cnt[i])
                GS_CHECK(cudaMemcpyAsync(cubes + off, acc_all[i], sizeof(uint64_t) * (size_t)acc_cnt[i],
                                         cudaMemcpyDeviceToDevice, st));
            off += acc_cnt[i];
            B.release(acc_all[i]);
        }
    }
    *cubes_out = cubes;
    *nc_out = nc;
    return GS_OK;
}

// backward request: dL/d(mesh vertices) in, dL/d(atoms, radii, D) out
struct BackReq {
    const double *gv;   // [nv, 3], host or device
    int64_t nv;
    double *g_atoms, *g_radii, *g_D;   // host or device
};

static int put_out(void *dst, const void *src, size_t bytes, cudaStream_t st);

// the batched form's per-molecule state entering mesh_impl: the prepared
// atoms (buffers owned by the batch), the accepted cubes of the shared level
// loop (mesh_impl takes them over) and the level statistics
struct PreMol {
    Prepared PR;
    uint64_t *cubes = nullptr;
    int64_t nc = 0;
    int64_t mismatches = 0;
    gs_stats lv;
};

// the level loop's fields of gs_stats (in the batched form those of the
// molecule's group, apart from the per-level decision counts)
static void copy_level_stats(gs_stats *d, const gs_stats &s)
{
    memcpy(d->examined, s.examined, sizeof(s.examined));
    memcpy(d->discarded, s.discarded, sizeof(s.discarded));
    memcpy(d->accepted, s.accepted, sizeof(s.accepted));
    memcpy(d->forced, s.forced, sizeof(s.forced));
    memcpy(d->split, s.split, sizeof(s.split));
    memcpy(d->ms_level, s.ms_level, sizeof(s.ms_level));
    d->pair_terms = s.pair_terms;
    d->atom_octets = s.atom_octets;
    d->recheck_cubes = s.recheck_cubes;
    d->recheck_bounds = s.recheck_bounds;
    d->recheck_precision = s.recheck_precision;
    d->recheck_zero = s.recheck_zero;
    d->recheck_rank = s.recheck_rank;
    d->estimate_fast_cubes = s.estimate_fast_cubes;
    d->mixed_err_ratio = s.mixed_err_ratio;
    d->mixed_band_ratio = s.mixed_band_ratio;
    d->ms_upload = s.ms_upload;
    d->ms_bin = s.ms_bin;
    d->ms_levels = s.ms_levels;
    d->ms_accum = s.ms_accum;
    d->n_accum_launches = s.n_accum_launches;
    d->retries = s.retries;
    for (int k = 0; k < 3; k++) d->near_threshold[k] = s.near_threshold[k];
}

static int mesh_impl(const double *atoms, const double *radii, int64_t n, double D, double c, double precision,
                     int max_depth, const gs_options &o, gs_mesh *out, cudaStream_t st, const BackReq *bw = nullptr,
                     gs_mesh_buffers *into = nullptr, int64_t chunk = (int64_t)1 << 21, bool *retryable = nullptr,
                     const PreMol *pre = nullptr)
{
    gs_stats local;
    gs_stats *stats = o.stats ? o.stats : &local;
    memset(stats, 0, sizeof(*stats));
    if (pre) copy_level_stats(stats, pre->lv);
    // the batch's cubes are this call's from here on: freed on an early
    // return, handed to the conformity pass below
    struct CubesGuard {
        uint64_t *p;
        cudaStream_t st;
        ~CubesGuard() { gs_free(p, st); }
    } pre_cubes{pre ? pre->cubes : nullptr, st};
    DevBufs B(st);
    Timer T(st);
    int tstart = T.mark();
    long long launches0 = gs_launch_count();
    unsigned *d_status = nullptr;
    // counters: [0..4] level decisions, [8] pairs, [9] vertex terms, [10..12] triangulation,
    // [13] rechecked cubes, [14] mismatches, [15..17] recheck reasons, [18] error-ratio bits
    unsigned long long *d_cnt = nullptr;
    int rc = B.get(&d_status, 1);
    if (!rc) rc = B.get(&d_cnt, GS_NCNT);
    if (rc) return rc;
    unsigned long long *d_near = nullptr;   // near-threshold counts (gs_stats.near_threshold)
    rc = B.get(&d_near, 4);
    if (rc) return rc;
    GS_CHECK(cudaMemsetAsync(d_status, 0, sizeof(unsigned), st));
    GS_CHECK(cudaMemsetAsync(d_cnt, 0, GS_NCNT * sizeof(unsigned long long), st));
    GS_CHECK(cudaMemsetAsync(d_near, 0, 4 * sizeof(unsigned long long), st));
    Prepared PR;
    if (pre) {
        PR = pre->PR;
    } else {
        NvtxRange nr("gs: upload, prep, cell list");
        rc = prepare(atoms, radii, n, D, c, o.cutoff_rel, precision, o.min_edge, max_depth, B, d_status, &PR, stats, T);
    }
    if (rc) return rc;
    PR.P.order = o.decision_order;
    PR.P.norm = o.precision_norm;
    PR.P.near = d_near;
    const GsProblem &P = PR.P;
    if (o.precision_mode == GS_PREC_MIXED) {
        rc = check_fp32_range(P);
        if (rc) return rc;
    }

    // ---- level loop (section 2.2, steps 1-3), or the batched form's result
    int tl0 = T.mark();
    uint64_t *cubes = nullptr;
    int64_t nc = 0;
    if (pre) {
        cubes = pre->cubes;
        nc = pre->nc;
    } else {
        rc = single_levels(P, o, max_depth, B, T, d_cnt, d_status, stats, chunk, retryable, &cubes, &nc);
        if (rc) return rc;
    }
    int tl1 = T.mark();

    // ---- cubes of different sizes (section 2.3, the points of neighbouring
    // cubes inside the current cube): with every accepted cube on one level
    // there is nothing to do
    int64_t splits = 0, agree_splits = 0;
    int acc_levels = 0;
    for (int l = 0; l <= max_depth; l++) acc_levels += (stats->accepted[l] + stats->forced[l]) > 0 ? 1 : 0;
    const bool constrain = acc_levels > 1 && o.conform_mode == GS_CONFORM_CONSTRAIN;
    NvtxRange nr_field("gs: conformity, lattice, field");
    pre_cubes.p = nullptr;
    if (acc_levels > 1) rc = gs_conformity(&cubes, &nc, max_depth, constrain ? 2 : 1, &splits, d_status, st);
    if (rc) { gs_free(cubes, st); return rc; }
    int tc1 = T.mark();

    // ---- lattice vertices, the field there (eq linear1's corner values)
    // and, for cubes of different sizes, the constrained values; a sign
    // disagreement splits the coarser cubes and the lattice is rebuilt, the
    // vertices it had keeping their field values
    const bool fp32 = o.precision_mode == GS_PREC_MIXED;
    uint64_t *vkeys = nullptr;
    int32_t *cvid = nullptr;
    int64_t nv = 0;
    double *phi = nullptr, *raw = nullptr;
    float *err = nullptr, *raw_err = nullptr;
    int64_t *mark = nullptr;
    GsHash hv{nullptr, nullptr, 0}, hc{nullptr, nullptr, 0};
    uint64_t *vslot = nullptr;
    GsCons K{nullptr, nullptr, nullptr, 0, 0, nullptr, {0}};
    uint8_t *mixed = nullptr;
    int64_t n_mixed = 0, nre = 0, ndw = 0;
    // after a round of splits: the new cubes (fresh), and the previous
    // lattice's raw field values and bounds for its nv_keep vertices, which
    // keep their ids in the extended lattice
    uint8_t *fresh = nullptr;
    double *raw_old = nullptr;
    float *err_old = nullptr;
    int64_t nv_keep = 0;
    auto release_all = [&](std::initializer_list<void *> ps) {
        for (void *q : ps) B.release(q);
    };
    B.keep(cubes);
    for (int iter = 0;; iter++) {
        if (iter > 64) return gs_fail(GS_ERR_CAPACITY, "cube sizes did not settle");
        if (!fresh) {
            rc = gs_lattice_vertices(cubes, nc, max_depth, &vkeys, &nv, &cvid, d_status, st, constrain ? &hv : nullptr,
                                     constrain ? &vslot : nullptr);
            B.keep(vkeys); B.keep(cvid); B.keep(hv.keys); B.keep(hv.vals); B.keep(vslot);
        } else {
            // after splits: the lattice grows by the new cubes' corners
            int64_t added = 0;
            B.forget(vkeys); B.forget(cvid);
            rc = gs_lattice_extend(cubes, nc, fresh, max_depth, hv, vslot, &vkeys, &nv, &cvid, &added, d_status, st);
            B.keep(vkeys); B.keep(cvid);
            B.release(fresh);
            fresh = nullptr;
        }
        if (rc) return rc;
        rc = B.get(&phi, (size_t)nv + 1);
        if (!rc && fp32) rc = B.get(&err, (size_t)nv + 1);
        if (!rc) rc = B.get(&mark, (size_t)nv + 1);
        if (rc) return rc;
        if (raw_old) {
            // the previous vertices keep their values and bounds, the new ones
            // (appended, ids nv_keep .. nv) are evaluated
            GS_CHECK(cudaMemcpyAsync(phi, raw_old, sizeof(double) * (size_t)nv_keep, cudaMemcpyDeviceToDevice, st));
            if (fp32)
                GS_CHECK(cudaMemcpyAsync(err, err_old, sizeof(float) * (size_t)nv_keep, cudaMemcpyDeviceToDevice, st));
            const int64_t nn = nv - nv_keep;
            if (nn > 0)
                rc = fp32 ? gs_field_f32(P, vkeys + nv_keep, nullptr, nn, phi + nv_keep, nullptr, err + nv_keep,
                                         d_cnt + 9, st)
                          : gs_field_f64(P, vkeys + nv_keep, nullptr, nn, phi + nv_keep, nullptr, d_cnt + 9, st);
            release_all({raw_old, err_old});
            raw_old = nullptr; err_old = nullptr;
        } else if (fp32) {
            rc = gs_field_f32(P, vkeys, nullptr, nv, phi, nullptr, err, d_cnt + 9, st);
        } else {
            rc = gs_field_f64(P, vkeys, nullptr, nv, phi, nullptr, d_cnt + 9, st);
        }
        if (!rc && fp32) {
            // where the inside test could depend on the FP32 error: double-word
            // FP32, and FP64 where that still leaves it open
            int64_t n1 = 0, n1b = 0;
            rc = gs_field_flag_near(P, phi, err, nv, mark, st);
            if (!rc) rc = gs_field_refine(P, vkeys, nv, mark, phi, err, &n1, &n1b, st);
            ndw += n1;
            nre += n1b;
        }
        if (rc) return rc;
        if (!constrain) break;
        rc = gs_hash_make(&hc, nc, st);
        if (rc) return rc;
        B.keep(hc.keys); B.keep(hc.vals);
        GS_LAUNCH(k_hash_index, (unsigned)((nc + 255) / 256), 256, 0, st)(hc, cubes, nc, d_status);
        rc = gs_cons_alloc(&K, nv, st);
        if (rc) return rc;
        B.keep(K.lev); B.keep(K.src); B.keep(K.t);
        rc = gs_cons_find(&K, hc, hv, vslot, vkeys, max_depth, nullptr, d_cnt + 26, d_status, st);
        B.keep(K.list);
        if (!rc && fp32 && K.ncons > 0) {
            // certain signs of the constrained values: their sources in FP64
            // where the interpolated bound leaves the side of c open
            double *psi = nullptr;
            float *epsi = nullptr;
            rc = B.get(&psi, (size_t)nv + 1);
            if (!rc) rc = B.get(&epsi, (size_t)nv + 1);
            if (!rc) {
                GS_CHECK(cudaMemcpyAsync(psi, phi, sizeof(double) * (size_t)nv, cudaMemcpyDeviceToDevice, st));
                GS_CHECK(cudaMemcpyAsync(epsi, err, sizeof(float) * (size_t)nv, cudaMemcpyDeviceToDevice, st));
                GS_CHECK(cudaMemsetAsync(mark, 0, sizeof(int64_t) * (size_t)(nv + 1), st));
                rc = gs_cons_apply(K, hc, vkeys, max_depth, P.c, psi, epsi, mark, nullptr, nullptr, d_cnt + 27, st);
            }
            if (!rc) rc = gs_cons_mark_up(K, max_depth, mark, st);
            if (!rc) rc = gs_cons_unmark(K, mark, st);
            int64_t n1 = 0, n1b = 0;
            if (!rc) rc = gs_field_refine(P, vkeys, nv, mark, phi, err, &n1, &n1b, st);
            ndw += n1;
            nre += n1b;
            if (!rc && n1 > n1b) {
                // FP64 for the sources whose refined bounds still leave a side open
                GS_CHECK(cudaMemcpyAsync(psi, phi, sizeof(double) * (size_t)nv, cudaMemcpyDeviceToDevice, st));
                GS_CHECK(cudaMemcpyAsync(epsi, err, sizeof(float) * (size_t)nv, cudaMemcpyDeviceToDevice, st));
                GS_CHECK(cudaMemsetAsync(mark, 0, sizeof(int64_t) * (size_t)(nv + 1), st));
                rc = gs_cons_apply(K, hc, vkeys, max_depth, P.c, psi, epsi, mark, nullptr, nullptr, d_cnt + 27, st);
                if (!rc) rc = gs_cons_mark_up(K, max_depth, mark, st);
                if (!rc) rc = gs_cons_unmark(K, mark, st);
                int64_t n1c = 0;
                if (!rc) rc = gs_field_recompute(P, vkeys, nv, mark, phi, err, &n1c, st);
                nre += n1c;
            }
            release_all({psi, epsi});
        }
        // the raw field values (and bounds), kept for a later round
        if (!rc) rc = B.get(&raw, (size_t)nv + 1);
        if (!rc && fp32) rc = B.get(&raw_err, (size_t)nv + 1);
        if (rc) return rc;
        GS_CHECK(cudaMemcpyAsync(raw, phi, sizeof(double) * (size_t)nv, cudaMemcpyDeviceToDevice, st));
        if (fp32) GS_CHECK(cudaMemcpyAsync(raw_err, err, sizeof(float) * (size_t)nv, cudaMemcpyDeviceToDevice, st));
        int64_t *split = nullptr;
        rc = B.get(&split, (size_t)nc + 1);
        if (!rc) rc = gs_fill_i64(split, nc, 1, st);
        int64_t nflip = 0;
        if (!rc) rc = gs_cons_apply(K, hc, vkeys, max_depth, P.c, phi, err, nullptr, split, &nflip, d_cnt + 27, st);
        if (!rc) rc = check_status(d_status, st, "constrained values");
        if (rc) return rc;
        if (nflip > 0) {
            int64_t ns = 0, ns2 = 0;
            B.forget(cubes);   // replaced (and freed) by the split
            rc = gs_split_counted(&cubes, &nc, split, &ns, st, &fresh);
            B.release(split);
            if (!rc) rc = gs_conformity(&cubes, &nc, max_depth, 2, &ns2, d_status, st, &fresh);
            B.keep(cubes); B.keep(fresh);
            if (rc) return rc;
            agree_splits += ns;
            splits += ns2;
            // this round's lattice grows into the next one's; its raw values
            // and bounds stay with its vertices
            raw_old = raw; err_old = raw_err; nv_keep = nv;
            release_all({phi, err, mark, hc.keys, hc.vals, K.lev, K.src, K.t, K.list});
            phi = nullptr; err = nullptr; mark = nullptr; raw = nullptr; raw_err = nullptr;
            hc = GsHash{nullptr, nullptr, 0};
            K = GsCons{nullptr, nullptr, nullptr, 0, 0, nullptr, {0}};
            continue;
        }
        release_all({split, raw, raw_err});
        raw = nullptr; raw_err = nullptr;
        rc = B.get(&mixed, (size_t)nc + 1);
        if (!rc) rc = gs_mixed_flags(K, cubes, nc, cvid, hv, vslot, max_depth, mixed, &n_mixed, d_cnt + 28, st);
        if (rc) return rc;
        break;
    }
    stats->constrained_vertices = K.ncons;
    stats->agreement_splits = agree_splits;
    stats->mixed_cubes = n_mixed;
    if (fp32) {
        // FP64 where a surface point's position (first-order bound 8e-6 A)
        // or a face or fold decision could depend on the FP32 error (the
        // constrained values carry their sources' interpolated bounds; a mark
        // on one passes to its sources, then the values are set again)
        GS_CHECK(cudaMemsetAsync(mark, 0, sizeof(int64_t) * (size_t)(nv + 1), st));
        TriCtx X;
        memset(&X, 0, sizeof(X));
        X.cubes = cubes; X.cvid = cvid; X.phi = phi; X.ncubes = nc; X.c = P.c;
        for (int a3 = 0; a3 < 3; a3++) X.origin[a3] = P.origin[a3];
        X.min_edge = P.min_edge; X.max_depth = P.max_depth;
        // first the double-word FP32 values (a bound some 1e4 times tighter),
        // then the same marks over the cubes that marked a corner, and FP64
        // for what they mark again (folds near a double root, mostly)
        int64_t *mlist = nullptr, nlist = 0;
        rc = B.get(&mlist, (size_t)nc + 1);
        if (!rc) rc = gs_tri_marks(X, err, 8e-6, mark, d_cnt + 32, nullptr, 0, mlist, &nlist, st);
        if (!rc && constrain) rc = gs_cons_mark_up(K, max_depth, mark, st);
        if (!rc && constrain) rc = gs_cons_unmark(K, mark, st);
        int64_t n2 = 0, n2b = 0;
        if (!rc) rc = gs_field_refine(P, vkeys, nv, mark, phi, err, &n2, &n2b, st);
        ndw += n2;
        nre += n2b;
        if (!rc && constrain)
            rc = gs_cons_apply(K, hc, vkeys, max_depth, P.c, phi, err, nullptr, nullptr, nullptr, d_cnt + 27, st);
        if (!rc && nlist > 0) {
            GS_CHECK(cudaMemsetAsync(mark, 0, sizeof(int64_t) * (size_t)(nv + 1), st));
            rc = gs_tri_marks(X, err, 8e-6, mark, d_cnt + 36, mlist, nlist, nullptr, nullptr, st);
            if (!rc && constrain) rc = gs_cons_mark_up(K, max_depth, mark, st);
            if (!rc && constrain) rc = gs_cons_unmark(K, mark, st);
            int64_t n3 = 0;
            if (!rc) rc = gs_field_recompute(P, vkeys, nv, mark, phi, err, &n3, st);
            nre += n3;
            if (!rc && constrain && n3 > 0)
                rc = gs_cons_apply(K, hc, vkeys, max_depth, P.c, phi, err, nullptr, nullptr, nullptr, d_cnt + 27, st);
        }
        B.release(mlist);
        stats->recheck_vertices = nre;
    }
    stats->refine_vertices = ndw;
    nr_field.end();
    if (rc) return rc;
    int tf1 = T.mark();

    // ---- triangulation and welding
    MeshDev M;
    M.cubes = cubes;
    M.nc = nc;
    MixInfo mx{n_mixed > 0 ? mixed : nullptr, hc, hv, vslot};
    rc = gs_count_near(phi, nv, P.c, d_near + 3, st);
    if (rc) return rc;
    {
        NvtxRange nr("gs: triangulate, weld");
        rc = surface_from_values(P, cubes, nc, cvid, phi, B, d_status, d_cnt + 10, M, stats, T, &mx);
    }
    if (rc) return rc;
    int tw1 = T.mark();
    if (bw) {
        // adjoint: dL/dp -> dL/dphi at the lattice vertices -> dL/d(atoms, radii, D)
        if (bw->nv != M.nv)
            return gs_fail(GS_ERR_ARG, "grad_vertices has %lld rows, the mesh %lld vertices", (long long)bw->nv,
                           (long long)M.nv);
        const double *gv = bw->gv;
        if (M.nv > 0 && !on_device(gv)) {
            double *tmp = nullptr;
            rc = B.get(&tmp, 3 * (size_t)M.nv);
            if (rc) return rc;
            GS_CHECK(cudaMemcpyAsync(tmp, gv, sizeof(double) * 3 * (size_t)M.nv, cudaMemcpyHostToDevice, st));
            gv = tmp;
        }
        double *lambda = nullptr, *g = nullptr;
        rc = B.get(&lambda, (size_t)nv + 1);
        if (!rc) rc = B.get(&g, 4 * (size_t)n + 1);
        if (rc) return rc;
        GS_CHECK(cudaMemsetAsync(g, 0, sizeof(double) * (4 * (size_t)n + 1), st));
        TriCtx X;
        memset(&X, 0, sizeof(X));
        X.cubes = cubes; X.cvid = cvid; X.phi = phi; X.ncubes = nc; X.c = P.c;
        for (int a3 = 0; a3 < 3; a3++) X.origin[a3] = P.origin[a3];
        X.min_edge = P.min_edge; X.max_depth = P.max_depth;
        rc = gs_vertex_adjoint(X, vkeys, nv, M.vkeys, gv, M.nv, lambda, d_status, st);
        // a constrained value passes its adjoint on to the corners it interpolates
        if (!rc && constrain) rc = gs_cons_adjoint(K, max_depth, lambda, st);
        if (!rc) rc = gs_field_adjoint(P, PR.perm, vkeys, lambda, nv, g, g + 3 * n, g + 4 * n, st);
        if (!rc) rc = check_status(d_status, st, "adjoint");
        if (!rc && bw->g_atoms) rc = put_out(bw->g_atoms, g, sizeof(double) * 3 * (size_t)n, st);
        if (!rc && bw->g_radii) rc = put_out(bw->g_radii, g + 3 * n, sizeof(double) * (size_t)n, st);
        if (!rc && bw->g_D) rc = put_out(bw->g_D, g + 4 * n, sizeof(double), st);
        if (rc) return rc;
        GS_CHECK(gs_sync(st));
    }
    if (out) {
        rc = into ? finish_into(M, into, st) : finish_output(M, o, out, st);
        if (rc) return rc;
    }
    int tend = T.mark();
    GS_CHECK(gs_sync(st));
    unsigned long long h[GS_NCNT], hn[4];
    GS_CHECK(cudaMemcpy(h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost));
    GS_CHECK(cudaMemcpy(hn, d_near, sizeof(hn), cudaMemcpyDeviceToHost));
    for (int k = 0; k < 4; k++) stats->near_threshold[k] = (int64_t)hn[k];
    stats->recheck_bounds = (int64_t)h[15];
    stats->recheck_precision = (int64_t)h[16];
    stats->recheck_zero = (int64_t)h[17];
    stats->recheck_rank = (int64_t)h[20];
    for (int k = 0; k < 3; k++) stats->vertex_mark_cubes[k] = (int64_t)h[32 + k];
    stats->vertex_mark_all = (int64_t)h[35];
    for (int k = 0; k < 3; k++) stats->vertex_mark_fp64_cubes[k] = (int64_t)h[36 + k];
    stats->estimate_fast_cubes = (int64_t)h[25];
    {
        unsigned bits = (unsigned)(h[18] & 0xffffffffull);
        float r;
        memcpy(&r, &bits, sizeof(r));
        stats->mixed_err_ratio = r;
        bits = (unsigned)(h[19] & 0xffffffffull);
        memcpy(&r, &bits, sizeof(r));
        stats->mixed_band_ratio = r;
    }
    stats->pair_terms = (int64_t)h[8];
    stats->atom_octets = (int64_t)h[24];
    stats->vertex_terms = (int64_t)h[9];
    stats->recheck_cubes = (int64_t)h[13];
    if (out) out->mismatches = (int64_t)h[14];
    stats->conformity_splits = splits;
    stats->n_cubes_final = nc;
    stats->n_lattice_vertices = nv;
    stats->n_vertices = M.nv;
    stats->n_triangles = M.nt;
    stats->ms_levels = T.ms(tl0, tl1);
    stats->ms_conformity = T.ms(tl1, tc1);
    stats->ms_field = T.ms(tc1, tf1);
    stats->ms_download = T.ms(tw1, tend);
    stats->ms_total = T.ms(tstart, tend);
    stats->n_kernel_launches = gs_launch_count() - launches0;
    if (pre) {
        copy_level_stats(stats, pre->lv);
        if (out) out->mismatches = pre->mismatches;
    }
    return GS_OK;
}

// mesh_impl, tried once more with level chunks of 2^18 octets (1/8 of the
// memory per chunk) when the level loop ran out of device memory or of an
// internal table
static int mesh_with_retry(const double *atoms, const double *radii, int64_t n, double D, double c, double precision,
                           int max_depth, const gs_options &o, gs_mesh *out, cudaStream_t st,
                           const BackReq *bw = nullptr, gs_mesh_buffers *into = nullptr)
{
    bool retry = false;
    int rc = mesh_impl(atoms, radii, n, D, c, precision, max_depth, o, out, st, bw, into, (int64_t)1 << 21, &retry);
    if (rc && retry) {
        cudaGetLastError();
        rc = mesh_impl(atoms, radii, n, D, c, precision, max_depth, o, out, st, bw, into, (int64_t)1 << 18);
        if (!rc && o.stats) o.stats->retries = 1;
    }
    return rc;
}

static int check_mesh_args(const double *atoms, const double *radii, int64_t n_atoms, double D, double c,
                           double precision, int max_depth, const gs_options &o)
{
    if (!atoms || !radii || n_atoms <= 0 || n_atoms > ((int64_t)1 << 31) - 1)
        return gs_fail(GS_ERR_ARG, "need 1 <= n_atoms < 2^31 and non-NULL inputs");
    if (!(D > 0) || !std::isfinite(D) || !(c > 0) || !std::isfinite(c) || !(precision > 0) || !std::isfinite(precision))
        return gs_fail(GS_ERR_ARG, "D, c and precision must be positive and finite");
    if (max_depth < 0 || max_depth > 20) return gs_fail(GS_ERR_ARG, "max_depth must be in [0, 20]");
    if (!(o.min_edge > 0) || !std::isfinite(o.min_edge)) return gs_fail(GS_ERR_ARG, "min_edge must be positive");
    if (!(o.cutoff_rel > 0 && o.cutoff_rel < 1)) return gs_fail(GS_ERR_ARG, "cutoff_rel must be in (0,1)");
    if (o.precision_mode != GS_PREC_FP64 && o.precision_mode != GS_PREC_MIXED)
        return gs_fail(GS_ERR_ARG, "unknown precision mode");
    if (o.child_mode != GS_CHILD_REPROJECT && o.child_mode != GS_CHILD_REEXPAND)
        return gs_fail(GS_ERR_ARG, "unknown child mode");
    if (o.child_mode == GS_CHILD_REEXPAND && o.precision_mode != GS_PREC_FP64)
        return gs_fail(GS_ERR_ARG, "child re-expansion is implemented in the FP64 form only");
    if (o.decision_order != GS_ORDER_BOUNDS_FIRST && o.decision_order != GS_ORDER_LITERAL)
        return gs_fail(GS_ERR_ARG, "unknown decision order");
    if (o.precision_norm != GS_NORM_SUM && o.precision_norm != GS_NORM_MAX && o.precision_norm != GS_NORM_RSS)
        return gs_fail(GS_ERR_ARG, "unknown precision norm");
    if (o.conform_mode != GS_CONFORM_CONSTRAIN && o.conform_mode != GS_CONFORM_EQUAL)
        return gs_fail(GS_ERR_ARG, "unknown conform mode");
    if ((o.decision_order != GS_ORDER_BOUNDS_FIRST || o.precision_norm != GS_NORM_SUM) &&
        o.precision_mode != GS_PREC_FP64)
        return gs_fail(GS_ERR_ARG, "the alternative decision order and norms are implemented in the FP64 form only");
    return GS_OK;
}

extern "C" int mesh_gaussian_surface(const double *atoms, const double *radii, int64_t n_atoms, double D, double c,
                                     double precision, int max_depth, const gs_options *opt, gs_mesh *out)
{
    if (!out) return gs_fail(GS_ERR_ARG, "out is NULL");
    memset(out, 0, sizeof(*out));
    gs_options o = opt ? *opt : gs_default_options();
    int rc = check_mesh_args(atoms, radii, n_atoms, D, c, precision, max_depth, o);
    if (rc) return rc;
    rc = device_setup();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)o.cuda_stream;
    bool own = false;
    if (!st) {
        GS_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        own = true;
    }
    rc = mesh_with_retry(atoms, radii, n_atoms, D, c, precision, max_depth, o, out, st);
    cudaError_t e = gs_sync(st);
    if (own) cudaStreamDestroy(st);
    if (!rc && e != cudaSuccess) rc = gs_fail_cuda(e, "stream", __FILE__, __LINE__);
    if (rc) mesh_free(out);
    return rc;
}

extern "C" int mesh_gaussian_surface_into(const double *atoms, const double *radii, int64_t n_atoms, double D,
                                          double c, double precision, int max_depth, const gs_options *opt,
                                          gs_mesh_buffers *out)
{
    if (!out) return gs_fail(GS_ERR_ARG, "out is NULL");
    out->n_vertices = out->n_triangles = out->n_cubes = 0;
    if (out->cap_vertices < 0 || out->cap_triangles < 0 || out->cap_cubes < 0 ||
        (out->cap_vertices > 0 && !out->vertices) || (out->cap_triangles > 0 && !out->triangles))
        return gs_fail(GS_ERR_ARG, "negative capacity or missing vertices/triangles buffer");
    gs_options o = opt ? *opt : gs_default_options();
    o.device_output = 1;   // the mesh stays on the device until it is copied into the buffers
    int rc = check_mesh_args(atoms, radii, n_atoms, D, c, precision, max_depth, o);
    if (rc) return rc;
    rc = device_setup();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)o.cuda_stream;
    bool own = false;
    if (!st) {
        GS_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        own = true;
    }
    gs_mesh unused;
    memset(&unused, 0, sizeof(unused));
    rc = mesh_with_retry(atoms, radii, n_atoms, D, c, precision, max_depth, o, &unused, st, nullptr, out);
    cudaError_t e = gs_sync(st);
    if (own) cudaStreamDestroy(st);
    if (!rc && e != cudaSuccess) rc = gs_fail_cuda(e, "stream", __FILE__, __LINE__);
    return rc;
}

// ---- the batched form

// the level loop of a group of molecules sharing D (section 2.2, steps 1-3,
// for all of them at once): each kernel of a level runs once over the
// octets of every molecule of the group.  On return pm[mols[g]] holds the
// molecule's accepted cubes, in the order its own level loop gives them,
// and its level statistics.
static int group_levels(const std::vector<int64_t> &mols, std::vector<PreMol> &pm, const gs_options &o,
                        int max_depth, cudaStream_t st, int64_t CH, bool *retryable)
{
    const int G = (int)mols.size();
    const int L = max_depth + 1;
    DevBufs B(st);
    Timer T(st);
    const int t0 = T.mark();
    unsigned *d_status = nullptr;
    unsigned long long *d_cnt = nullptr, *d_molcnt = nullptr;
    GsProblem *d_probs = nullptr;
    int rc = B.get(&d_status, 1);
    if (!rc) rc = B.get(&d_cnt, GS_NCNT);
    if (!rc) rc = B.get(&d_molcnt, 5 * (size_t)G);
    if (!rc) rc = B.get(&d_probs, (size_t)G);
    unsigned long long *d_near = nullptr;
    if (!rc) rc = B.get(&d_near, 4);
    if (rc) return rc;
    GS_CHECK(cudaMemsetAsync(d_near, 0, 4 * sizeof(unsigned long long), st));
    std::vector<GsProblem> hp((size_t)G);
    for (int g = 0; g < G; g++) hp[(size_t)g] = pm[(size_t)mols[(size_t)g]].PR.P;
    GS_CHECK(cudaMemsetAsync(d_status, 0, sizeof(unsigned), st));
    GS_CHECK(cudaMemsetAsync(d_cnt, 0, GS_NCNT * sizeof(unsigned long long), st));
    GS_CHECK(cudaMemcpyAsync(d_probs, hp.data(), sizeof(GsProblem) * (size_t)G, cudaMemcpyHostToDevice, st));
    // the record the shared kernels read: the group's common scalars (D, c,
    // precision, depth, order, norm); level-0 children outside a molecule's
    // root grid are masked explicitly, so its root extent is unbounded
    GsProblem P0 = hp[0];
    for (int a = 0; a < 3; a++) P0.nroot[a] = (int64_t)1 << 40;
    P0.near = d_near;
    uint64_t *parents = nullptr;
    uint8_t *vmask0 = nullptr;
    int32_t *pmol = nullptr;
    int64_t n_oct = 0;
    rc = gs_root_blocks_batch(hp.data(), G, &parents, &vmask0, &pmol, &n_oct, st);
    if (rc) return rc;
    B.keep(parents); B.keep(vmask0); B.keep(pmol);
    std::vector<std::vector<uint64_t *>> acc((size_t)L);
    std::vector<std::vector<int32_t *>> accm((size_t)L);
    std::vector<std::vector<int64_t>> accn((size_t)L);
    std::vector<int64_t> molcnt((size_t)L * 5 * (size_t)G, 0);
    gs_stats gst;
    memset(&gst, 0, sizeof(gst));
    for (int l = 0; l < L && n_oct > 0; l++) {
        char lname[48];
        snprintf(lname, sizeof(lname), "gs: batch level %d", l);
        NvtxRange nr(lname);
        const int ta = T.mark();
        GS_CHECK(cudaMemsetAsync(d_cnt, 0, 5 * sizeof(unsigned long long), st));
        GS_CHECK(cudaMemsetAsync(d_molcnt, 0, 5 * (size_t)G * sizeof(unsigned long long), st));
        LevelBatch lb;
        lb.d_probs = d_probs;
        lb.pmol = pmol;
        lb.pvmask = l == 0 ? vmask0 : nullptr;
        lb.molcnt = d_molcnt;
        uint64_t *next = nullptr;
        int64_t nn = 0;
        rc = run_level(P0, l, parents, n_oct, o.precision_mode, B, acc[(size_t)l], accn[(size_t)l], &next, &nn, d_cnt,
                       d_cnt + 8, d_cnt + 13, d_cnt + 14, (o.debug_flags & 1) != 0, d_status, &gst, false, nullptr,
                       nullptr, (o.debug_flags & 2) ? (int64_t)1000 : CH, &lb);
        for (auto q : acc[(size_t)l]) B.keep(q);
        for (auto q : lb.acc_mol) B.keep(q);
        accm[(size_t)l] = lb.acc_mol;
        B.release(parents); B.release(pmol);
        if (l == 0) B.release(vmask0);
        if (rc) {
            if (retryable && (rc == GS_ERR_OOM || rc == GS_ERR_CAPACITY)) *retryable = true;
            gs_free(next, st);
            gs_free(lb.next_mol, st);
            return rc;
        }
        parents = next;
        pmol = lb.next_mol;
        B.keep(parents); B.keep(pmol);
        n_oct = nn;
        const int tb = T.mark();
        std::vector<unsigned long long> h((size_t)G * 5 + 5);
        GS_CHECK(cudaMemcpyAsync(h.data(), d_molcnt, sizeof(unsigned long long) * 5 * (size_t)G,
                                 cudaMemcpyDeviceToHost, st));
        GS_CHECK(cudaMemcpyAsync(h.data() + 5 * (size_t)G, d_cnt, 5 * sizeof(unsigned long long),
                                 cudaMemcpyDeviceToHost, st));
        GS_CHECK(gs_sync(st));
        for (size_t k = 0; k < 5 * (size_t)G; k++) molcnt[(size_t)l * 5 * G + k] = (int64_t)h[k];
        const unsigned long long *tot = h.data() + 5 * (size_t)G;
        gst.examined[l] = (int64_t)tot[0]; gst.discarded[l] = (int64_t)tot[1]; gst.accepted[l] = (int64_t)tot[2];
        gst.forced[l] = (int64_t)tot[3]; gst.split[l] = (int64_t)tot[4];
        gst.ms_level[l] = T.ms(ta, tb);
    }
    B.release(parents); B.release(pmol);
    rc = check_status(d_status, st, "levels");
    if (rc) return rc;
    // each molecule's accepted cubes, level by level: per level the parts
    // are grouped by molecule, molecule g's run starting at the sum of the
    // earlier molecules' counts
    auto nacc = [&](int l, int g) {
        const int64_t *m = &molcnt[((size_t)l * G + (size_t)g) * 5];
        return m[2] + m[3];
    };
    std::vector<int64_t> shift((size_t)L * G), ntot((size_t)G, 0);
    for (int l = 0; l < L; l++) {
        int64_t seg = 0, parts = 0;
        for (int g = 0; g < G; g++) {
            shift[(size_t)l * G + g] = ntot[(size_t)g] - seg;
            seg += nacc(l, g);
            ntot[(size_t)g] += nacc(l, g);
        }
        for (auto v : accn[(size_t)l]) parts += v;
        if (parts != seg) return gs_fail(GS_ERR_DEVICE_STATUS, "level %d: %lld accepted cubes, %lld by molecule", l,
                                         (long long)parts, (long long)seg);
    }
    std::vector<uint64_t *> outs((size_t)G, nullptr);
    auto drop_outs = [&]() {
        for (auto q : outs) gs_free(q, st);
    };
    for (int g = 0; g < G && !rc; g++) rc = gs_alloc((void **)&outs[(size_t)g], sizeof(uint64_t) * (size_t)(ntot[(size_t)g] + 1), st);
    int64_t *d_shift = nullptr, *d_cap = nullptr;
    uint64_t **d_outs = nullptr;
    if (!rc) rc = B.get(&d_shift, shift.size());
    if (!rc) rc = B.get(&d_cap, (size_t)G);
    if (!rc) rc = B.get(&d_outs, (size_t)G);
    if (rc) { drop_outs(); return rc; }
    GS_CHECK(cudaMemcpyAsync(d_shift, shift.data(), sizeof(int64_t) * shift.size(), cudaMemcpyHostToDevice, st));
    GS_CHECK(cudaMemcpyAsync(d_cap, ntot.data(), sizeof(int64_t) * (size_t)G, cudaMemcpyHostToDevice, st));
    GS_CHECK(cudaMemcpyAsync(d_outs, outs.data(), sizeof(uint64_t *) * (size_t)G, cudaMemcpyHostToDevice, st));
    for (int l = 0; l < L && !rc; l++) {
        int64_t q0 = 0;
        for (size_t p = 0; p < acc[(size_t)l].size() && !rc; p++) {
            rc = gs_scatter_cubes(acc[(size_t)l][p], accm[(size_t)l][p], accn[(size_t)l][p], q0,
                                  d_shift + (size_t)l * G, d_outs, d_cap, d_status, st);
            q0 += accn[(size_t)l][p];
        }
    }
    if (!rc) rc = check_status(d_status, st, "batch cubes");
    const int t1 = T.mark();
    unsigned long long h[GS_NCNT], hn[4];
    cudaError_t e = cudaMemcpyAsync(h, d_cnt, sizeof(h), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = cudaMemcpyAsync(hn, d_near, sizeof(hn), cudaMemcpyDeviceToHost, st);
    if (e == cudaSuccess) e = gs_sync(st);
    if (!rc && e != cudaSuccess) rc = gs_fail_cuda(e, "batch levels", __FILE__, __LINE__);
    if (rc) { drop_outs(); return rc; }
    gst.pair_terms = (int64_t)h[8];
    gst.atom_octets = (int64_t)h[24];
    gst.recheck_cubes = (int64_t)h[13];
    gst.recheck_bounds = (int64_t)h[15];
    gst.recheck_precision = (int64_t)h[16];
    gst.recheck_zero = (int64_t)h[17];
    gst.recheck_rank = (int64_t)h[20];
    gst.estimate_fast_cubes = (int64_t)h[25];
    {
        unsigned bits = (unsigned)(h[18] & 0xffffffffull);
        float r;
        memcpy(&r, &bits, sizeof(r));
        gst.mixed_err_ratio = r;
        bits = (unsigned)(h[19] & 0xffffffffull);
        memcpy(&r, &bits, sizeof(r));
        gst.mixed_band_ratio = r;
    }
    gst.ms_levels = T.ms(t0, t1);
    for (int k = 0; k < 3; k++) gst.near_threshold[k] = (int64_t)hn[k];
    for (int g = 0; g < G; g++) {
        PreMol &q = pm[(size_t)mols[(size_t)g]];
        q.lv = gst;
        for (int l = 0; l < L; l++) {
            const int64_t *m = &molcnt[((size_t)l * G + (size_t)g) * 5];
            q.lv.examined[l] = m[0]; q.lv.discarded[l] = m[1]; q.lv.accepted[l] = m[2];
            q.lv.forced[l] = m[3]; q.lv.split[l] = m[4];
        }
        q.cubes = outs[(size_t)g];
        q.nc = ntot[(size_t)g];
        q.mismatches = (int64_t)h[14];
    }
    return GS_OK;
}

// one host thread per worker, each with its own stream, runs whole
// single-molecule meshes, largest molecules first
static int batch_threads(const double *atoms, const double *radii, const int64_t *offsets, int64_t n_mols,
                         const double *D, double c, double precision, int max_depth, const gs_options &base,
                         int n_workers, gs_mesh *out, gs_stats *stats, std::vector<PreMol> *pm)
{
    int dev = 0;
    GS_CHECK(cudaGetDevice(&dev));
    std::vector<int64_t> order((size_t)n_mols);
    for (int64_t m = 0; m < n_mols; m++) order[(size_t)m] = m;
    std::stable_sort(order.begin(), order.end(), [&](int64_t a, int64_t b) {
        if (pm) return (*pm)[(size_t)a].nc > (*pm)[(size_t)b].nc;
        return offsets[a + 1] - offsets[a] > offsets[b + 1] - offsets[b];
    });
    std::atomic<int64_t> next{0};
    std::mutex mu;
    int first_rc = 0;
    int64_t first_mol = -1;
    std::string first_msg;
    auto worker = [&]() {
        cudaStream_t st = nullptr;
        if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            std::lock_guard<std::mutex> lk(mu);
            if (!first_rc) { first_rc = GS_ERR_CUDA; first_msg = "stream creation failed"; }
            return;
        }
        for (;;) {
            int64_t t = next.fetch_add(1);
            if (t >= n_mols) break;
            const int64_t m = order[(size_t)t], o0 = offsets[m], n = offsets[m + 1] - o0;
            gs_options o = base;
            o.cuda_stream = st;
            o.stats = stats ? &stats[m] : nullptr;
            int r;
            if (pm) {
                r = mesh_impl(atoms + 3 * o0, radii + o0, n, D[m], c, precision, max_depth, o, &out[m], st, nullptr,
                              nullptr, (int64_t)1 << 21, nullptr, &(*pm)[(size_t)m]);
                (*pm)[(size_t)m].cubes = nullptr;   // handed over
            } else {
                r = mesh_with_retry(atoms + 3 * o0, radii + o0, n, D[m], c, precision, max_depth, o, &out[m], st);
            }
            cudaError_t e = gs_sync(st);
            if (!r && e != cudaSuccess) r = gs_fail_cuda(e, "stream", __FILE__, __LINE__);
            if (r) {
                std::lock_guard<std::mutex> lk(mu);
                if (!first_rc) { first_rc = r; first_mol = m; first_msg = gs_last_error(); }
            }
        }
        cudaStreamDestroy(st);
    };
    int nw = n_workers < 1 ? 1 : n_workers;
    if (nw > n_mols) nw = (int)n_mols;
    std::vector<std::thread> pool;
    for (int w = 1; w < nw; w++) pool.emplace_back(worker);
    worker();
    for (auto &th : pool) th.join();
    if (first_rc) return gs_fail(first_rc, "molecule %lld: %s", (long long)first_mol, first_msg.c_str());
    return GS_OK;
}

// shared level loops, pipelined: one host thread per group of molecules
// with equal D prepares them (atoms uploaded, cell list) and runs the
// group's level loop on its own stream, then hands the molecules to the
// workers, which finish each mesh (conformity, lattice, field,
// triangulation, weld) on their own streams, largest first.  A group's
// meshes are finished while the next group's levels run.
static int batch_shared(const double *atoms, const double *radii, const int64_t *offsets, int64_t n_mols,
                        const double *D, double c, double precision, int max_depth, const gs_options &base,
                        int n_workers, gs_mesh *out, gs_stats *stats)
{
    // groups of equal D, in order of first appearance
    std::vector<std::vector<int64_t>> groups;
    std::vector<int> group_of((size_t)n_mols);
    {
        std::vector<double> keys;
        for (int64_t m = 0; m < n_mols; m++) {
            size_t k = 0;
            while (k < keys.size() && keys[k] != D[m]) k++;
            if (k == keys.size()) { keys.push_back(D[m]); groups.emplace_back(); }
            groups[k].push_back(m);
            group_of[(size_t)m] = (int)k;
        }
    }
    const int NG = (int)groups.size();
    int dev = 0;
    GS_CHECK(cudaGetDevice(&dev));
    std::vector<cudaStream_t> gstream((size_t)NG, nullptr);
    for (int k = 0; k < NG; k++) {
        cudaError_t e = cudaStreamCreateWithFlags(&gstream[(size_t)k], cudaStreamNonBlocking);
        if (e != cudaSuccess) {
            for (int j = 0; j < k; j++) cudaStreamDestroy(gstream[(size_t)j]);
            return gs_fail_cuda(e, "stream", __FILE__, __LINE__);
        }
    }
    std::vector<PreMol> pm((size_t)n_mols);
    std::vector<std::vector<std::unique_ptr<DevBufs>>> bufs((size_t)NG);
    std::mutex mu;
    std::condition_variable cv;
    std::vector<int64_t> ready;
    int groups_left = NG;
    bool failed = false;
    int first_rc = 0;
    int64_t first_mol = -1;
    std::string first_msg;
    auto fail = [&](int r, int64_t m) {
        std::lock_guard<std::mutex> lk(mu);
        if (!first_rc) { first_rc = r; first_mol = m; first_msg = gs_last_error(); }
        failed = true;
        cv.notify_all();
    };
    auto group_job = [&](int k) {
        cudaStream_t st = gstream[(size_t)k];
        int rc = cudaSetDevice(dev) == cudaSuccess ? GS_OK : gs_fail(GS_ERR_CUDA, "cudaSetDevice failed");
        int64_t bad = -1;
        {
            DevBufs B(st);
            unsigned *d_status = nullptr;
            if (!rc) rc = B.get(&d_status, 1);
            if (!rc) {
                cudaError_t e = cudaMemsetAsync(d_status, 0, sizeof(unsigned), st);
                if (e != cudaSuccess) rc = gs_fail_cuda(e, "status", __FILE__, __LINE__);
            }
            Timer T(st);
            for (int64_t m : groups[(size_t)k]) {
                if (rc) break;
                const int64_t o0 = offsets[m], n = offsets[m + 1] - o0;
                bufs[(size_t)k].emplace_back(new DevBufs(st));
                NvtxRange nr("gs: batch prepare");
                rc = prepare(atoms + 3 * o0, radii + o0, n, D[m], c, base.cutoff_rel, precision, base.min_edge,
                             max_depth, *bufs[(size_t)k].back(), d_status, &pm[(size_t)m].PR, nullptr, T);
                if (!rc) {
                    pm[(size_t)m].PR.P.order = base.decision_order;
                    pm[(size_t)m].PR.P.norm = base.precision_norm;
                    if (base.precision_mode == GS_PREC_MIXED) rc = check_fp32_range(pm[(size_t)m].PR.P);
                }
                if (rc) bad = m;
            }
        }
        if (!rc) {
            bool retry = false;
            rc = group_levels(groups[(size_t)k], pm, base, max_depth, st, (int64_t)1 << 21, &retry);
            if (rc && retry) {
                cudaGetLastError();
                rc = group_levels(groups[(size_t)k], pm, base, max_depth, st, (int64_t)1 << 18, nullptr);
                if (!rc)
                    for (int64_t m : groups[(size_t)k]) pm[(size_t)m].lv.retries = 1;
            }
        }
        if (!rc) {
            cudaError_t e = gs_sync(st);
            if (e != cudaSuccess) rc = gs_fail_cuda(e, "batch levels", __FILE__, __LINE__);
        }
        if (rc) { fail(rc, bad); }
        std::lock_guard<std::mutex> lk(mu);
        if (!rc) ready.insert(ready.end(), groups[(size_t)k].begin(), groups[(size_t)k].end());
        groups_left--;
        cv.notify_all();
    };
    auto worker = [&]() {
        cudaStream_t st = nullptr;
        if (cudaSetDevice(dev) != cudaSuccess || cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking) != cudaSuccess) {
            fail(gs_fail(GS_ERR_CUDA, "worker stream creation failed"), -1);
            return;
        }
        for (;;) {
            int64_t m = -1;
            {
                std::unique_lock<std::mutex> lk(mu);
                cv.wait(lk, [&] { return failed || !ready.empty() || groups_left == 0; });
                if (failed || ready.empty()) break;
                // the largest mesh waiting
                size_t best = 0;
                for (size_t i = 1; i < ready.size(); i++)
                    if (pm[(size_t)ready[i]].nc > pm[(size_t)ready[best]].nc) best = i;
                m = ready[best];
                ready.erase(ready.begin() + (std::ptrdiff_t)best);
            }
            const int64_t o0 = offsets[m], n = offsets[m + 1] - o0;
            gs_options o = base;
            o.cuda_stream = st;
            o.stats = stats ? &stats[m] : nullptr;
            int r = mesh_impl(atoms + 3 * o0, radii + o0, n, D[m], c, precision, max_depth, o, &out[m], st, nullptr,
                              nullptr, (int64_t)1 << 21, nullptr, &pm[(size_t)m]);
            pm[(size_t)m].cubes = nullptr;   // handed over
            cudaError_t e = gs_sync(st);
            if (!r && e != cudaSuccess) r = gs_fail_cuda(e, "stream", __FILE__, __LINE__);
            if (r) fail(r, m);
        }
        cudaStreamDestroy(st);
    };
    int nw = n_workers < 1 ? 1 : n_workers;
    if (nw > n_mols) nw = (int)n_mols;
    {
        std::vector<std::thread> pool;
        for (int k = 0; k < NG; k++) pool.emplace_back(group_job, k);
        for (int w = 0; w < nw; w++) pool.emplace_back(worker);
        for (auto &th : pool) th.join();
    }
    // cubes not handed to a worker, then the prepared atoms, on the streams
    // they were made on (every worker has waited for its own stream)
    for (int64_t m = 0; m < n_mols; m++) gs_free(pm[(size_t)m].cubes, gstream[(size_t)group_of[(size_t)m]]);
    bufs.clear();
    cudaError_t e = cudaSuccess;
    for (auto st : gstream) {
        cudaError_t e2 = cudaStreamSynchronize(st);
        if (e == cudaSuccess) e = e2;
        cudaStreamDestroy(st);
    }
    if (first_rc) {
        if (first_mol >= 0) return gs_fail(first_rc, "molecule %lld: %s", (long long)first_mol, first_msg.c_str());
        return gs_fail(first_rc, "%s", first_msg.c_str());
    }
    if (e != cudaSuccess) return gs_fail_cuda(e, "stream", __FILE__, __LINE__);
    return GS_OK;
}

extern "C" int mesh_gaussian_surface_batch(const double *atoms, const double *radii, const int64_t *offsets,
                                           int64_t n_mols, const double *D, double c, double precision, int max_depth,
                                           const gs_options *opt, int n_workers, gs_mesh *out, gs_stats *stats)
{
    if (!out || n_mols <= 0 || !offsets || !D) return gs_fail(GS_ERR_ARG, "need n_mols >= 1, offsets, D and out");
    for (int64_t m = 0; m < n_mols; m++) memset(&out[m], 0, sizeof(gs_mesh));
    gs_options base = opt ? *opt : gs_default_options();
    if (offsets[0] != 0) return gs_fail(GS_ERR_ARG, "offsets[0] must be 0");
    if (base.batch_mode != GS_BATCH_SHARED_LEVELS && base.batch_mode != GS_BATCH_THREADS)
        return gs_fail(GS_ERR_ARG, "unknown batch mode");
    for (int64_t m = 0; m < n_mols; m++) {
        if (offsets[m + 1] <= offsets[m]) return gs_fail(GS_ERR_ARG, "molecule %lld is empty", (long long)m);
        int rc = check_mesh_args(atoms, radii, offsets[m + 1] - offsets[m], D[m], c, precision, max_depth, base);
        if (rc) return rc;
    }
    int rc = device_setup();
    if (rc) return rc;
    // re-expanded child tensors follow each molecule's own parents: no shared loop
    const bool shared = base.batch_mode == GS_BATCH_SHARED_LEVELS && base.child_mode != GS_CHILD_REEXPAND;
    if (stats)
        for (int64_t m = 0; m < n_mols; m++) memset(&stats[m], 0, sizeof(gs_stats));
    rc = shared ? batch_shared(atoms, radii, offsets, n_mols, D, c, precision, max_depth, base, n_workers, out, stats)
                : batch_threads(atoms, radii, offsets, n_mols, D, c, precision, max_depth, base, n_workers, out, stats,
                                nullptr);
    if (rc)
        for (int64_t m = 0; m < n_mols; m++) mesh_free(&out[m]);
    return rc;
}

extern "C" int gs_mesh_backward(const double *atoms, const double *radii, int64_t n_atoms, double D, double c,
                                double precision, int max_depth, const gs_options *opt, const double *grad_vertices,
                                int64_t n_vertices, double *grad_atoms, double *grad_radii, double *grad_D)
{
    gs_options o = opt ? *opt : gs_default_options();
    int rc = check_mesh_args(atoms, radii, n_atoms, D, c, precision, max_depth, o);
    if (rc) return rc;
    if (n_vertices < 0 || (n_vertices > 0 && !grad_vertices))
        return gs_fail(GS_ERR_ARG, "grad_vertices is NULL");
    rc = device_setup();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)o.cuda_stream;
    bool own = false;
    if (!st) {
        GS_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        own = true;
    }
    BackReq bw;
    bw.gv = grad_vertices;
    bw.nv = n_vertices;
    bw.g_atoms = grad_atoms;
    bw.g_radii = grad_radii;
    bw.g_D = grad_D;
    rc = mesh_with_retry(atoms, radii, n_atoms, D, c, precision, max_depth, o, nullptr, st, &bw);
    cudaError_t e = gs_sync(st);
    if (own) cudaStreamDestroy(st);
    if (!rc && e != cudaSuccess) rc = gs_fail_cuda(e, "stream", __FILE__, __LINE__);
    return rc;
}

static int put_in(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    GS_CHECK(cudaMemcpyAsync(dst, src, bytes, cudaMemcpyHostToDevice, st));
    return GS_OK;
}

__global__ void k_check_tri(const int32_t *t, int64_t n3, int64_t nv, unsigned *status)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n3 && (t[i] < 0 || t[i] >= nv)) atomicOr(status, 1u);
}

// every triangle index must name a vertex (the kernels read without checks)
static int check_tri_ids(const int32_t *d_t, int64_t nt, int64_t nv, unsigned *d_status, cudaStream_t st)
{
    GS_CHECK(cudaMemsetAsync(d_status, 0, sizeof(unsigned), st));
    GS_LAUNCH(k_check_tri, (unsigned)((3 * nt + 255) / 256), 256, 0, st)(d_t, 3 * nt, nv, d_status);
    unsigned h = 0;
    GS_CHECK(cudaMemcpyAsync(&h, d_status, sizeof(h), cudaMemcpyDeviceToHost, st));
    GS_CHECK(gs_sync(st));
    return h ? gs_fail(GS_ERR_ARG, "a triangle index is outside [0, n_vertices)") : GS_OK;
}

extern "C" int gs_mesh_intersections(const double *vertices, int64_t n_vertices, const int32_t *triangles,
                                     int64_t n_triangles, double tol, int64_t *n_pairs, const gs_options *opt)
{
    gs_options o = opt ? *opt : gs_default_options();
    if (!n_pairs || n_vertices < 0 || n_triangles < 0 || (n_vertices > 0 && !vertices) ||
        (n_triangles > 0 && !triangles) || n_vertices > ((int64_t)1 << 31) || !(tol >= 0.0))
        return gs_fail(GS_ERR_ARG, "bad arguments");
    *n_pairs = 0;
    int rc = device_setup();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)o.cuda_stream;
    bool own = false;
    if (!st) {
        GS_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        own = true;
    }
    {
        DevBufs B(st);
        const double *v = vertices;
        const int32_t *t = triangles;
        unsigned *d_status = nullptr;
        rc = B.get(&d_status, 1);
        if (!rc && n_vertices && !on_device(vertices)) {
            double *tv = nullptr;
            rc = B.get(&tv, 3 * (size_t)n_vertices);
            if (!rc) rc = put_in(tv, vertices, sizeof(double) * 3 * (size_t)n_vertices, st);
            v = tv;
        }
        if (!rc && n_triangles && !on_device(triangles)) {
            int32_t *tt = nullptr;
            rc = B.get(&tt, 3 * (size_t)n_triangles);
            if (!rc) rc = put_in(tt, triangles, sizeof(int32_t) * 3 * (size_t)n_triangles, st);
            t = tt;
        }
        if (!rc && n_triangles) rc = check_tri_ids(t, n_triangles, n_vertices, d_status, st);
        if (!rc) rc = gs_count_intersections(v, n_vertices, t, n_triangles, tol, n_pairs, st);
        cudaError_t e = gs_sync(st);
        if (!rc && e != cudaSuccess) rc = gs_fail_cuda(e, "stream", __FILE__, __LINE__);
    }
    if (own) cudaStreamDestroy(st);
    return rc;
}

extern "C" int gs_volume_area(const double *vertices, int64_t n_vertices, const int32_t *triangles,
                              int64_t n_triangles, double *volume_area, double *grad_volume, double *grad_area,
                              const gs_options *opt)
{
    gs_options o = opt ? *opt : gs_default_options();
    if (n_vertices < 0 || n_triangles < 0 || !volume_area || (n_vertices > 0 && !vertices) ||
        (n_triangles > 0 && !triangles) || n_vertices > ((int64_t)1 << 31))
        return gs_fail(GS_ERR_ARG, "bad arguments");
    int rc = device_setup();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)o.cuda_stream;
    bool own = false;
    if (!st) {
        GS_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking));
        own = true;
    }
    {
        DevBufs B(st);
        const double *v = vertices;
        const int32_t *t = triangles;
        double *acc = nullptr, *gV = nullptr, *gA = nullptr;
        unsigned *d_status = nullptr;
        rc = B.get(&acc, 2);
        if (!rc) rc = B.get(&d_status, 1);
        if (!rc && n_vertices && !on_device(vertices)) {
            double *tv = nullptr;
            rc = B.get(&tv, 3 * (size_t)n_vertices);
            if (!rc) rc = put_in(tv, vertices, sizeof(double) * 3 * (size_t)n_vertices, st);
            v = tv;
        }
        if (!rc && n_triangles && !on_device(triangles)) {
            int32_t *tt = nullptr;
            rc = B.get(&tt, 3 * (size_t)n_triangles);
            if (!rc) rc = put_in(tt, triangles, sizeof(int32_t) * 3 * (size_t)n_triangles, st);
            t = tt;
        }
        if (!rc && n_triangles) rc = check_tri_ids(t, n_triangles, n_vertices, d_status, st);
        if (!rc && grad_volume) rc = B.get(&gV, 3 * (size_t)n_vertices + 1);
        if (!rc && grad_area) rc = B.get(&gA, 3 * (size_t)n_vertices + 1);
        if (!rc && gV) GS_CHECK(cudaMemsetAsync(gV, 0, sizeof(double) * 3 * (size_t)n_vertices, st));
        if (!rc && gA) GS_CHECK(cudaMemsetAsync(gA, 0, sizeof(double) * 3 * (size_t)n_vertices, st));
        if (!rc) rc = gs_volume_area_dev(v, t, n_triangles, acc, gV, gA, st);
        if (!rc) rc = put_out(volume_area, acc, 2 * sizeof(double), st);
        if (!rc && gV) rc = put_out(grad_volume, gV, sizeof(double) * 3 * (size_t)n_vertices, st);
        if (!rc && gA) rc = put_out(grad_area, gA, sizeof(double) * 3 * (size_t)n_vertices, st);
        cudaError_t e = gs_sync(st);
        if (!rc && e != cudaSuccess) rc = gs_fail_cuda(e, "stream", __FILE__, __LINE__);
    }
    if (own) cudaStreamDestroy(st);
    return rc;
}

extern "C" int gs_triangulate_grid(int64_t nx, int64_t ny, int64_t nz, const double *values, double c,
                                   const gs_options *opt, gs_mesh *out)
{
    if (!out) return gs_fail(GS_ERR_ARG, "out is NULL");
    memset(out, 0, sizeof(*out));
    if (!values || nx <= 0 || ny <= 0 || nz <= 0 || nx > 4096 || ny > 4096 || nz > 4096)
        return gs_fail(GS_ERR_ARG, "grid dimensions must be in [1, 4096]");
    gs_options o = opt ? *opt : gs_default_options();
    int rc = device_setup();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)o.cuda_stream;
    bool own = false;
    if (!st) { GS_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)); own = true; }
    {
        DevBufs B(st);
        Timer T(st);
        gs_stats local;
        gs_stats *stats = o.stats ? o.stats : &local;
        memset(stats, 0, sizeof(*stats));
        GsProblem P;
        memset(&P, 0, sizeof(P));
        P.c = c; P.min_edge = 1.0; P.max_depth = 0;
        int64_t nvals = (nx + 1) * (ny + 1) * (nz + 1), nc = nx * ny * nz;
        const double *d_vals = values;
        unsigned *d_status = nullptr;
        unsigned long long *d_cnt = nullptr;
        uint64_t *cubes = nullptr;
        rc = B.get(&d_status, 1);
        if (!rc) rc = B.get(&d_cnt, 16);
        if (!rc) rc = B.get(&cubes, (size_t)nc);
        if (!rc && !on_device(values)) {
            double *p;
            rc = B.get(&p, (size_t)nvals);
            if (!rc) {
                cudaError_t e = cudaMemcpyAsync(p, values, sizeof(double) * (size_t)nvals, cudaMemcpyHostToDevice, st);
                if (e != cudaSuccess) rc = gs_fail_cuda(e, "grid upload", __FILE__, __LINE__);
            }
            d_vals = p;
        }
        if (!rc) {
            cudaMemsetAsync(d_status, 0, sizeof(unsigned), st);
            cudaMemsetAsync(d_cnt, 0, 16 * sizeof(unsigned long long), st);
            GS_LAUNCH(k_grid_cubes, (unsigned)((nc + 255) / 256), 256, 0, st)(nx, ny, nz, cubes);
        }
        uint64_t *vkeys = nullptr;
        int32_t *cvid = nullptr;
        int64_t nv = 0;
        if (!rc) rc = gs_lattice_vertices(cubes, nc, 0, &vkeys, &nv, &cvid, d_status, st);
        B.keep(vkeys); B.keep(cvid);
        double *phi = nullptr;
        if (!rc) rc = B.get(&phi, (size_t)nv + 1);
        if (!rc) GS_LAUNCH(k_fill_grid_phi, (unsigned)((nv + 255) / 256), 256, 0, st)(vkeys, nv, d_vals, nx, ny, phi);
        MeshDev M;
        M.cubes = cubes; M.nc = nc;
        if (!rc) rc = surface_from_values(P, cubes, nc, cvid, phi, B, d_status, d_cnt + 10, M, stats, T);
        if (!rc) rc = finish_output(M, o, out, st);
        if (!rc) { stats->n_vertices = M.nv; stats->n_triangles = M.nt; stats->n_cubes_final = nc; }
    }
    cudaError_t e = gs_sync(st);
    if (own) cudaStreamDestroy(st);
    if (!rc && e != cudaSuccess) rc = gs_fail_cuda(e, "stream", __FILE__, __LINE__);
    if (rc) mesh_free(out);
    return rc;
}

// copy a device result back where the caller wants it
static int put_out(void *dst, const void *src, size_t bytes, cudaStream_t st)
{
    if (!dst || !bytes) return GS_OK;
    GS_CHECK(cudaMemcpyAsync(dst, src, bytes, on_device(dst) ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost, st));
    return GS_OK;
}

extern "C" int gs_eval_field(const double *atoms, const double *radii, int64_t n_atoms, double D, double c,
                             double cutoff_rel, const double *points, int64_t n_points, double *phi, double *grad,
                             int precision_mode, void *stream)
{
    if (!atoms || !radii || n_atoms <= 0 || n_atoms >= ((int64_t)1 << 31) || n_points < 0 || (n_points && (!points || !phi)))
        return gs_fail(GS_ERR_ARG, "bad sizes or NULL pointers");
    if (!(D > 0) || !(c > 0) || !(cutoff_rel > 0 && cutoff_rel < 1)) return gs_fail(GS_ERR_ARG, "bad D, c or cutoff");
    if (precision_mode != GS_PREC_FP64 && precision_mode != GS_PREC_MIXED) return gs_fail(GS_ERR_ARG, "bad mode");
    int rc = device_setup();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    bool own = false;
    if (!st) { GS_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)); own = true; }
    {
        DevBufs B(st);
        Timer T(st);
        unsigned *d_status = nullptr;
        rc = B.get(&d_status, 1);
        if (!rc) { cudaMemsetAsync(d_status, 0, sizeof(unsigned), st); }
        Prepared PR;
        if (!rc) rc = prepare(atoms, radii, n_atoms, D, c, cutoff_rel, 1.0, 0.25, 0, B, d_status, &PR, nullptr, T);
        if (!rc && precision_mode == GS_PREC_MIXED) rc = check_fp32_range(PR.P);
        const double *d_pts = points;
        double *d_phi = nullptr, *d_grad = nullptr;
        if (!rc && n_points > 0) {
            if (!on_device(points)) {
                double *p;
                rc = B.get(&p, 3 * (size_t)n_points);
                if (!rc) {
                    cudaError_t e = cudaMemcpyAsync(p, points, sizeof(double) * 3 * (size_t)n_points, cudaMemcpyHostToDevice, st);
                    if (e != cudaSuccess) rc = gs_fail_cuda(e, "points upload", __FILE__, __LINE__);
                }
                d_pts = p;
            }
            if (!rc) rc = B.get(&d_phi, (size_t)n_points);
            if (!rc && grad) rc = B.get(&d_grad, 3 * (size_t)n_points);
            // points may lie outside the root grid: the cell list clamps them to its border cells
            if (!rc) {
                if (precision_mode == GS_PREC_FP64) rc = gs_field_f64(PR.P, nullptr, d_pts, n_points, d_phi, d_grad, nullptr, st);
                else rc = gs_field_f32(PR.P, nullptr, d_pts, n_points, d_phi, d_grad, nullptr, nullptr, st);
            }
            if (!rc) rc = put_out(phi, d_phi, sizeof(double) * (size_t)n_points, st);
            if (!rc && grad) rc = put_out(grad, d_grad, sizeof(double) * 3 * (size_t)n_points, st);
        }
        if (!rc) rc = check_status(d_status, st, "field");
    }
    cudaError_t e = gs_sync(st);
    if (own) cudaStreamDestroy(st);
    if (!rc && e != cudaSuccess) rc = gs_fail_cuda(e, "stream", __FILE__, __LINE__);
    return rc;
}

extern "C" int gs_eval_field_bounded(const double *atoms, const double *radii, int64_t n_atoms, double D, double c,
                                     double cutoff_rel, const double *points, int64_t n_points, double *phi,
                                     float *err, void *stream)
{
    if (!atoms || !radii || n_atoms <= 0 || n_atoms >= ((int64_t)1 << 31) || n_points < 0 ||
        (n_points && (!points || !phi || !err)))
        return gs_fail(GS_ERR_ARG, "bad sizes or NULL pointers");
    if (!(D > 0) || !(c > 0) || !(cutoff_rel > 0 && cutoff_rel < 1)) return gs_fail(GS_ERR_ARG, "bad D, c or cutoff");
    int rc = device_setup();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    bool own = false;
    if (!st) { GS_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)); own = true; }
    {
        DevBufs B(st);
        Timer T(st);
        unsigned *d_status = nullptr;
        rc = B.get(&d_status, 1);
        if (!rc) { cudaMemsetAsync(d_status, 0, sizeof(unsigned), st); }
        Prepared PR;
        if (!rc) rc = prepare(atoms, radii, n_atoms, D, c, cutoff_rel, 1.0, 0.25, 0, B, d_status, &PR, nullptr, T);
        if (!rc) rc = check_fp32_range(PR.P);
        if (!rc && n_points > 0) {
            const double *d_pts = points;
            double *d_phi = nullptr;
            float *d_err = nullptr;
            if (!on_device(points)) {
                double *q;
                rc = B.get(&q, 3 * (size_t)n_points);
                if (!rc) rc = gs_copy_from_host(q, points, sizeof(double) * 3 * (size_t)n_points, st);
                d_pts = q;
            }
            if (!rc) rc = B.get(&d_phi, (size_t)n_points);
            if (!rc) rc = B.get(&d_err, (size_t)n_points);
            if (!rc) rc = gs_field_dw(PR.P, nullptr, d_pts, n_points, d_phi, d_err, nullptr, st);
            if (!rc) rc = put_out(phi, d_phi, sizeof(double) * (size_t)n_points, st);
            if (!rc) rc = put_out(err, d_err, sizeof(float) * (size_t)n_points, st);
        }
        if (!rc) rc = check_status(d_status, st, "field");
    }
    cudaError_t e = gs_sync(st);
    if (own) cudaStreamDestroy(st);
    if (!rc && e != cudaSuccess) rc = gs_fail_cuda(e, "stream", __FILE__, __LINE__);
    return rc;
}

extern "C" int gs_cube_decisions(const double *atoms, const double *radii, int64_t n_atoms, double D, double c,
                                 double precision, double min_edge, int max_depth, double cutoff_rel,
                                 const uint64_t *cube_keys, int64_t n_cubes, double *A, double *bounds, int32_t *dec,
                                 int precision_mode, void *stream)
{
    if (!atoms || !radii || n_atoms <= 0 || n_atoms >= ((int64_t)1 << 31) || n_cubes < 0 || (n_cubes && (!cube_keys || !dec)))
        return gs_fail(GS_ERR_ARG, "bad sizes or NULL pointers");
    if (!(D > 0) || !(c > 0) || !(precision > 0) || !(min_edge > 0) || max_depth < 0 || max_depth > 20 ||
        !(cutoff_rel > 0 && cutoff_rel < 1))
        return gs_fail(GS_ERR_ARG, "bad parameters");
    (void)precision_mode;
    int rc = device_setup();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    bool own = false;
    if (!st) { GS_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)); own = true; }
    {
        DevBufs B(st);
        Timer T(st);
        unsigned *d_status = nullptr;
        rc = B.get(&d_status, 1);
        if (!rc) cudaMemsetAsync(d_status, 0, sizeof(unsigned), st);
        Prepared PR;
        if (!rc) rc = prepare(atoms, radii, n_atoms, D, c, cutoff_rel, precision, min_edge, max_depth, B, d_status, &PR, nullptr, T);
        // group by level; each cube becomes its own octet with one valid child
        std::vector<uint64_t> hk((size_t)n_cubes);
        if (!rc && n_cubes) {
            cudaError_t e = cudaMemcpyAsync(hk.data(), cube_keys, sizeof(uint64_t) * (size_t)n_cubes,
                                            on_device(cube_keys) ? cudaMemcpyDeviceToHost : cudaMemcpyHostToHost, st);
            if (e == cudaSuccess) e = gs_sync(st);
            if (e != cudaSuccess) rc = gs_fail_cuda(e, "keys", __FILE__, __LINE__);
        }
        std::vector<double> hA, hB;
        std::vector<int32_t> hD((size_t)n_cubes);
        if (A) hA.resize((size_t)n_cubes * 64);
        if (bounds) hB.resize((size_t)n_cubes * 6);
        for (int l = 0; l <= max_depth && !rc; l++) {
            std::vector<int64_t> idx;
            std::vector<uint64_t> par;
            std::vector<uint8_t> vm;
            for (int64_t i = 0; i < n_cubes; i++)
                if ((int)gk_level(hk[i]) == l) {
                    uint64_t k = hk[i];
                    idx.push_back(i);
                    par.push_back(gk_make(gk_x(k) >> 1, gk_y(k) >> 1, gk_z(k) >> 1, GT_CUBE, l > 0 ? l - 1 : 0));
                    vm.push_back((uint8_t)(1u << ((gk_x(k) & 1) | ((gk_y(k) & 1) << 1) | ((gk_z(k) & 1) << 2))));
                }
            int64_t m = (int64_t)idx.size();
            if (!m) continue;
            uint64_t *dp; uint8_t *dv, *dd; double *dA, *dB;
            rc = B.get(&dp, (size_t)m);
            if (!rc) rc = B.get(&dv, (size_t)m);
            if (!rc) rc = B.get(&dd, (size_t)m * 8);
            if (!rc) rc = B.get(&dA, (size_t)m * 8 * 64);
            if (!rc) rc = B.get(&dB, (size_t)m * 8 * 6);
            if (rc) break;
            cudaMemcpyAsync(dp, par.data(), sizeof(uint64_t) * (size_t)m, cudaMemcpyHostToDevice, st);
            cudaMemcpyAsync(dv, vm.data(), (size_t)m, cudaMemcpyHostToDevice, st);
            rc = gs_accum_f64(PR.P, l, dp, dv, m, dA, nullptr, d_status, st);
            if (!rc) rc = gs_estimate_f64(PR.P, l, dA, m * 8, dp, dv, dd, dB, st);
            std::vector<double> tA((size_t)m * 8 * 64), tB((size_t)m * 8 * 6);
            std::vector<uint8_t> tD((size_t)m * 8);
            if (!rc) {
                cudaMemcpyAsync(tA.data(), dA, sizeof(double) * tA.size(), cudaMemcpyDeviceToHost, st);
                cudaMemcpyAsync(tB.data(), dB, sizeof(double) * tB.size(), cudaMemcpyDeviceToHost, st);
                cudaMemcpyAsync(tD.data(), dd, tD.size(), cudaMemcpyDeviceToHost, st);
                cudaError_t e = gs_sync(st);
                if (e != cudaSuccess) rc = gs_fail_cuda(e, "decisions", __FILE__, __LINE__);
            }
            for (int64_t t = 0; t < m && !rc; t++) {
                int ch = __builtin_ctz(vm[t]);
                int64_t q = 8 * t + ch, i = idx[t];
                hD[i] = tD[q];
                if (A) memcpy(&hA[64 * i], &tA[64 * q], 64 * sizeof(double));
                if (bounds) memcpy(&hB[6 * i], &tB[6 * q], 6 * sizeof(double));
            }
        }
        if (!rc) rc = check_status(d_status, st, "decisions");
        if (!rc && n_cubes) {
            bool ddev = on_device(dec);
            cudaMemcpyKind k = ddev ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost;
            cudaMemcpy(dec, hD.data(), sizeof(int32_t) * (size_t)n_cubes, k);
            if (A) cudaMemcpy(A, hA.data(), sizeof(double) * hA.size(), on_device(A) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost);
            if (bounds) cudaMemcpy(bounds, hB.data(), sizeof(double) * hB.size(), on_device(bounds) ? cudaMemcpyHostToDevice : cudaMemcpyHostToHost);
        }
    }
    cudaError_t e = gs_sync(st);
    if (own) cudaStreamDestroy(st);
    if (!rc && e != cudaSuccess) rc = gs_fail_cuda(e, "stream", __FILE__, __LINE__);
    return rc;
}

extern "C" int gs_bin_atoms(const double *atoms, int64_t n_atoms, double cell_size, const double *origin,
                            const int64_t *dims, int32_t *cell_start, int32_t *atom_perm, void *stream)
{
    if (!atoms || n_atoms <= 0 || n_atoms >= ((int64_t)1 << 31) || !(cell_size > 0) || !origin || !dims ||
        !cell_start || !atom_perm)
        return gs_fail(GS_ERR_ARG, "bad arguments");
    int cd[3];
    int64_t ncell = 1;
    for (int a = 0; a < 3; a++) {
        if (dims[a] <= 0 || dims[a] > (1 << 20)) return gs_fail(GS_ERR_ARG, "bad dims");
        cd[a] = (int)dims[a];
        ncell *= dims[a];
    }
    if (ncell >= ((int64_t)1 << 31)) return gs_fail(GS_ERR_ARG, "too many cells");
    int rc = device_setup();
    if (rc) return rc;
    cudaStream_t st = (cudaStream_t)stream;
    bool own = false;
    if (!st) { GS_CHECK(cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking)); own = true; }
    {
        DevBufs B(st);
        const double *d_xyz = atoms;
        if (!on_device(atoms)) {
            double *p;
            rc = B.get(&p, 3 * (size_t)n_atoms);
            if (!rc) cudaMemcpyAsync(p, atoms, sizeof(double) * 3 * (size_t)n_atoms, cudaMemcpyHostToDevice, st);
            d_xyz = p;
        }
        int32_t *cs, *pm;
        if (!rc) rc = B.get(&cs, (size_t)ncell + 1);
        if (!rc) rc = B.get(&pm, (size_t)n_atoms);
        if (!rc) rc = gs_build_cells(d_xyz, n_atoms, origin, cell_size, cd, cs, pm, st);
        if (!rc) rc = put_out(cell_start, cs, sizeof(int32_t) * (size_t)(ncell + 1), st);
        if (!rc) rc = put_out(atom_perm, pm, sizeof(int32_t) * (size_t)n_atoms, st);
    }
    cudaError_t e = gs_sync(st);
    if (own) cudaStreamDestroy(st);
    if (!rc && e != cudaSuccess) rc = gs_fail_cuda(e, "stream", __FILE__, __LINE__);
    return rc;
}
