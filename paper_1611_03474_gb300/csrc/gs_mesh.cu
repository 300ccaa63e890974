// gs_mesh.cu -- hash-table passes around the triangulation:
//   * conformity: an accepted cube touching a finer accepted cube along a
//     face or an edge is split into 8 accepted children until no such
//     contact remains (the paper's rule that points of neighbouring cubes
//     inside the current cube are considered, section 2.3, realised by
//     equalising sizes across every shared face and edge);
//   * lattice vertices of the accepted cubes with deterministic ids (owner =
//     smallest (cube, corner) index, then a prefix sum in cube order);
//   * same-size face neighbours of each cube;
//   * welding of the emitted surface points by key (owner = first copy),
//     and remapping of the triangles' keys to vertex ids.
#include "gs_host.cuh"

__global__ void k_hash_clear(uint64_t *keys, uint64_t *vals, uint64_t cap, uint64_t vinit)
{
    for (uint64_t i = (uint64_t)blockIdx.x * blockDim.x + threadIdx.x; i < cap; i += (uint64_t)gridDim.x * blockDim.x) {
        keys[i] = GS_EMPTY;
        if (vals) vals[i] = vinit;
    }
}

int gs_hash_make(GsHash *H, int64_t n, cudaStream_t st)
{
    uint64_t cap = 1024;
    while (cap < (uint64_t)(2 * n + 16)) cap <<= 1;
    H->mask = cap - 1;
    H->keys = nullptr; H->vals = nullptr;
    int rc = gs_alloc((void **)&H->keys, sizeof(uint64_t) * cap, st);
    if (!rc) rc = gs_alloc((void **)&H->vals, sizeof(uint64_t) * cap, st);
    if (rc) { gs_free(H->keys, st); gs_free(H->vals, st); H->keys = H->vals = nullptr; return rc; }
    GS_LAUNCH(k_hash_clear, 1024, 256, 0, st)(H->keys, H->vals, cap, ~0ull);
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

void gs_hash_free(GsHash *H, cudaStream_t st)
{
    gs_free(H->keys, st);
    gs_free(H->vals, st);
    H->keys = H->vals = nullptr;
}

// insert keys[i] with value i (keys unique)
__global__ void k_hash_index(GsHash H, const uint64_t *keys, int64_t n, unsigned *status)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    int64_t s = gs_hash_insert(H, keys[i], status);
    if (s >= 0) H.vals[s] = (uint64_t)i;
}

// ---------------------------------------------------------------- conformity
// Each accepted cube F marks every coarser accepted cube C that contains one
// of F's 18 face or edge neighbour cells: exactly the cubes that touch a
// finer accepted cube along a face or an edge.
__global__ void k_conform_mark(GsHash H, const uint64_t *cubes, int64_t n, int64_t *cnt)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = cubes[i];
    int lf = (int)gk_level(k);
    if (lf == 0) return;
    int64_t x = gk_x(k), y = gk_y(k), z = gk_z(k);
    for (int d = 0; d < 27; d++) {
        int dx = d % 3 - 1, dy = (d / 3) % 3 - 1, dz = d / 9 - 1;
        int nz_ = (dx != 0) + (dy != 0) + (dz != 0);
        if (nz_ == 0 || nz_ == 3) continue;
        int64_t X = x + dx, Y = y + dy, Z = z + dz;
        if (X < 0 || Y < 0 || Z < 0) continue;
        for (int l = lf - 1; l >= 0; l--) {
            int sh = lf - l;
            int64_t s = gs_hash_find(H, gk_make(X >> sh, Y >> sh, Z >> sh, GT_CUBE, (unsigned)l));
            if (s >= 0) {
                cnt[H.vals[s]] = 8;
                break;
            }
        }
    }
}

__global__ void k_fill_one(int64_t *cnt, int64_t n)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) cnt[i] = 1;
}

__global__ void k_conform_emit(const uint64_t *cubes, int64_t n, const int64_t *off, uint64_t *out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = cubes[i];
    int64_t o = off[i], m = off[i + 1] - off[i];
    if (m == 1) { out[o] = k; return; }
    unsigned l = gk_level(k) + 1;
    int64_t x = gk_x(k), y = gk_y(k), z = gk_z(k);
    for (int c = 0; c < 8; c++) out[o + c] = gk_make(2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + (c >> 2), GT_CUBE, l);
}

// in/out: *d_cubes (replaced when split), *n
int gs_conformity(uint64_t **d_cubes, int64_t *n, int max_depth, int64_t *splits, unsigned *d_status, cudaStream_t st)
{
    *splits = 0;
    for (int pass = 0; pass < 64; pass++) {
        int64_t m = *n;
        if (m == 0) return GS_OK;
        GsHash H;
        int rc = gs_hash_make(&H, m, st);
        if (rc) return rc;
        unsigned nb = (unsigned)((m + 255) / 256);
        GS_LAUNCH(k_hash_index, nb, 256, 0, st)(H, *d_cubes, m, d_status);
        int64_t *cnt = nullptr, *tot = nullptr;
        rc = gs_alloc((void **)&cnt, sizeof(int64_t) * (size_t)(m + 1), st);
        if (!rc) rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
        if (rc) { gs_hash_free(&H, st); gs_free(cnt, st); return rc; }
        cudaMemsetAsync(cnt + m, 0, sizeof(int64_t), st);
        GS_LAUNCH(k_fill_one, nb, 256, 0, st)(cnt, m);
        GS_LAUNCH(k_conform_mark, nb, 256, 0, st)(H, *d_cubes, m, cnt);
        gs_hash_free(&H, st);
        rc = gs_scan_i64(cnt, m + 1, tot, st);
        int64_t total = 0;
        if (!rc) {
            cudaError_t e = cudaMemcpyAsync(&total, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
            if (e == cudaSuccess) e = cudaStreamSynchronize(st);
            if (e != cudaSuccess) rc = gs_fail_cuda(e, "conformity count", __FILE__, __LINE__);
        }
        if (rc || total == m) { gs_free(cnt, st); gs_free(tot, st); return rc; }
        uint64_t *out = nullptr;
        rc = gs_alloc((void **)&out, sizeof(uint64_t) * (size_t)total, st);
        if (rc) { gs_free(cnt, st); gs_free(tot, st); return rc; }
        GS_LAUNCH(k_conform_emit, nb, 256, 0, st)(*d_cubes, m, cnt, out);
        gs_free(cnt, st); gs_free(tot, st);
        gs_free(*d_cubes, st);
        *d_cubes = out;
        *splits += (total - m) / 7;
        *n = total;
    }
    return gs_fail(GS_ERR_CAPACITY, "conformity did not converge");
}

// ---------------------------------------------------------------- lattice vertices
__device__ __forceinline__ uint64_t corner_key(uint64_t ck, int v, int max_depth)
{
    int64_t s = (int64_t)1 << (max_depth - (int)gk_level(ck));
    return gk_make((gk_x(ck) + (v & 1)) * s, (gk_y(ck) + ((v >> 1) & 1)) * s, (gk_z(ck) + (v >> 2)) * s, GT_VERT, 0);
}

__global__ void k_vert_claim(GsHash H, const uint64_t *cubes, int64_t n, int max_depth, unsigned *status)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 8) return;
    uint64_t key = corner_key(cubes[t >> 3], (int)(t & 7), max_depth);
    int64_t s = gs_hash_insert(H, key, status);
    if (s >= 0) atomicMin((unsigned long long *)&H.vals[s], (unsigned long long)t);
}

__global__ void k_vert_owner(GsHash H, const uint64_t *cubes, int64_t n, int max_depth, int64_t *flag)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 8) return;
    uint64_t key = corner_key(cubes[t >> 3], (int)(t & 7), max_depth);
    int64_t s = gs_hash_find(H, key);
    flag[t] = (s >= 0 && H.vals[s] == (uint64_t)t) ? 1 : 0;
}

__global__ void k_vert_write(GsHash H, const uint64_t *cubes, int64_t n, int max_depth, const int64_t *off,
                             uint64_t *vkeys, uint64_t *slot_id)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 8) return;
    if (off[t + 1] == off[t]) return;
    uint64_t key = corner_key(cubes[t >> 3], (int)(t & 7), max_depth);
    int64_t s = gs_hash_find(H, key);
    vkeys[off[t]] = key;
    if (s >= 0) slot_id[s] = (uint64_t)off[t];
}

__global__ void k_vert_cvid(GsHash H, const uint64_t *cubes, int64_t n, int max_depth, const uint64_t *slot_id,
                            int32_t *cvid, unsigned *status)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 8) return;
    uint64_t key = corner_key(cubes[t >> 3], (int)(t & 7), max_depth);
    int64_t s = gs_hash_find(H, key);
    if (s < 0) { atomicOr(status, GS_ST_LOOKUP); cvid[t] = 0; return; }
    cvid[t] = (int32_t)slot_id[s];
}

int gs_lattice_vertices(const uint64_t *d_cubes, int64_t n, int max_depth, uint64_t **d_vkeys, int64_t *nv,
                        int32_t **d_cvid, unsigned *d_status, cudaStream_t st)
{
    *d_vkeys = nullptr; *d_cvid = nullptr; *nv = 0;
    if (n <= 0) return GS_OK;
    int64_t m = n * 8;
    GsHash H;
    int rc = gs_hash_make(&H, m / 2 + 8, st);
    if (rc) return rc;
    int64_t *flag = nullptr, *tot = nullptr;
    uint64_t *slot_id = nullptr;
    rc = gs_alloc((void **)&flag, sizeof(int64_t) * (size_t)(m + 1), st);
    if (!rc) rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
    if (!rc) rc = gs_alloc((void **)&slot_id, sizeof(uint64_t) * (size_t)(H.mask + 1), st);
    unsigned nb = (unsigned)((m + 255) / 256);
    if (!rc) {
        GS_LAUNCH(k_vert_claim, nb, 256, 0, st)(H, d_cubes, n, max_depth, d_status);
        cudaMemsetAsync(flag + m, 0, sizeof(int64_t), st);
        GS_LAUNCH(k_vert_owner, nb, 256, 0, st)(H, d_cubes, n, max_depth, flag);
        rc = gs_scan_i64(flag, m + 1, tot, st);
    }
    int64_t total = 0;
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(&total, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = gs_fail_cuda(e, "vertex count", __FILE__, __LINE__);
    }
    if (!rc) rc = gs_alloc((void **)d_vkeys, sizeof(uint64_t) * (size_t)(total + 1), st);
    if (!rc) rc = gs_alloc((void **)d_cvid, sizeof(int32_t) * (size_t)m, st);
    if (!rc) {
        GS_LAUNCH(k_vert_write, nb, 256, 0, st)(H, d_cubes, n, max_depth, flag, *d_vkeys, slot_id);
        GS_LAUNCH(k_vert_cvid, nb, 256, 0, st)(H, d_cubes, n, max_depth, slot_id, *d_cvid, d_status);
    }
    gs_free(flag, st); gs_free(tot, st); gs_free(slot_id, st);
    gs_hash_free(&H, st);
    if (rc) { gs_free(*d_vkeys, st); gs_free(*d_cvid, st); *d_vkeys = nullptr; *d_cvid = nullptr; return rc; }
    GS_CHECK(cudaGetLastError());
    *nv = total;
    return GS_OK;
}

// ---------------------------------------------------------------- face neighbours
__global__ void k_neighbours(GsHash H, const uint64_t *cubes, int64_t n, int32_t *nbr)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 6) return;
    int64_t i = t / 6;
    int f = (int)(t % 6), a = f >> 1, sd = f & 1;
    uint64_t k = cubes[i];
    int64_t c[3] = {gk_x(k), gk_y(k), gk_z(k)};
    c[a] += sd ? 1 : -1;
    int32_t r = -1;
    if (c[a] >= 0 && c[a] <= (int64_t)GK_MASK) {
        int64_t s = gs_hash_find(H, gk_make(c[0], c[1], c[2], GT_CUBE, gk_level(k)));
        if (s >= 0) r = (int32_t)H.vals[s];
    }
    nbr[t] = r;
}

int gs_neighbours(const uint64_t *d_cubes, int64_t n, int32_t **d_nbr, unsigned *d_status, cudaStream_t st)
{
    *d_nbr = nullptr;
    if (n <= 0) return GS_OK;
    GsHash H;
    int rc = gs_hash_make(&H, n, st);
    if (rc) return rc;
    GS_LAUNCH(k_hash_index, (unsigned)((n + 255) / 256), 256, 0, st)(H, d_cubes, n, d_status);
    rc = gs_alloc((void **)d_nbr, sizeof(int32_t) * 6 * (size_t)n, st);
    if (!rc) GS_LAUNCH(k_neighbours, (unsigned)((6 * n + 255) / 256), 256, 0, st)(H, d_cubes, n, *d_nbr);
    gs_hash_free(&H, st);
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// ---------------------------------------------------------------- weld
__global__ void k_weld_claim(GsHash H, const uint64_t *pk, int64_t n, unsigned *status)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int64_t s = gs_hash_insert(H, pk[t], status);
    if (s >= 0) atomicMin((unsigned long long *)&H.vals[s], (unsigned long long)t);
}
__global__ void k_weld_owner(GsHash H, const uint64_t *pk, int64_t n, int64_t *flag)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int64_t s = gs_hash_find(H, pk[t]);
    flag[t] = (s >= 0 && H.vals[s] == (uint64_t)t) ? 1 : 0;
}
__global__ void k_weld_write(GsHash H, const uint64_t *pk, const double *pxyz, int64_t n, const int64_t *off,
                             uint64_t *vkeys, double *vxyz, uint64_t *slot_id)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    if (off[t + 1] == off[t]) return;
    int64_t id = off[t];
    vkeys[id] = pk[t];
    vxyz[3 * id] = pxyz[3 * t];
    vxyz[3 * id + 1] = pxyz[3 * t + 1];
    vxyz[3 * id + 2] = pxyz[3 * t + 2];
    int64_t s = gs_hash_find(H, pk[t]);
    if (s >= 0) slot_id[s] = (uint64_t)id;
}
__global__ void k_weld_tris(GsHash H, const uint64_t *slot_id, const uint64_t *tk, int64_t ntri, int32_t *tri,
                            unsigned *status)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= 3 * ntri) return;
    int64_t s = gs_hash_find(H, tk[t]);
    if (s < 0) { atomicOr(status, GS_ST_LOOKUP); tri[t] = 0; return; }
    tri[t] = (int32_t)slot_id[s];
}

int gs_weld(const uint64_t *d_pk, const double *d_pxyz, int64_t npt, const uint64_t *d_tk, int64_t ntri,
            uint64_t **d_vkeys, double **d_vxyz, int64_t *nv, int32_t **d_tri, unsigned *d_status, cudaStream_t st)
{
    *d_vkeys = nullptr; *d_vxyz = nullptr; *d_tri = nullptr; *nv = 0;
    if (npt <= 0) return GS_OK;
    GsHash H;
    int rc = gs_hash_make(&H, npt / 2 + 8, st);
    if (rc) return rc;
    int64_t *flag = nullptr, *tot = nullptr;
    uint64_t *slot_id = nullptr;
    rc = gs_alloc((void **)&flag, sizeof(int64_t) * (size_t)(npt + 1), st);
    if (!rc) rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
    if (!rc) rc = gs_alloc((void **)&slot_id, sizeof(uint64_t) * (size_t)(H.mask + 1), st);
    unsigned nb = (unsigned)((npt + 255) / 256);
    if (!rc) {
        GS_LAUNCH(k_weld_claim, nb, 256, 0, st)(H, d_pk, npt, d_status);
        cudaMemsetAsync(flag + npt, 0, sizeof(int64_t), st);
        GS_LAUNCH(k_weld_owner, nb, 256, 0, st)(H, d_pk, npt, flag);
        rc = gs_scan_i64(flag, npt + 1, tot, st);
    }
    int64_t total = 0;
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(&total, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = cudaStreamSynchronize(st);
        if (e != cudaSuccess) rc = gs_fail_cuda(e, "weld count", __FILE__, __LINE__);
    }
    if (!rc) rc = gs_alloc((void **)d_vkeys, sizeof(uint64_t) * (size_t)(total + 1), st);
    if (!rc) rc = gs_alloc((void **)d_vxyz, sizeof(double) * 3 * (size_t)(total + 1), st);
    if (!rc) rc = gs_alloc((void **)d_tri, sizeof(int32_t) * 3 * (size_t)(ntri + 1), st);
    if (!rc) {
        GS_LAUNCH(k_weld_write, nb, 256, 0, st)(H, d_pk, d_pxyz, npt, flag, *d_vkeys, *d_vxyz, slot_id);
        if (ntri > 0)
            GS_LAUNCH(k_weld_tris, (unsigned)((3 * ntri + 255) / 256), 256, 0, st)(H, slot_id, d_tk, ntri, *d_tri, d_status);
    }
    gs_free(flag, st); gs_free(tot, st); gs_free(slot_id, st);
    gs_hash_free(&H, st);
    if (rc) {
        gs_free(*d_vkeys, st); gs_free(*d_vxyz, st); gs_free(*d_tri, st);
        *d_vkeys = nullptr; *d_vxyz = nullptr; *d_tri = nullptr;
        return rc;
    }
    GS_CHECK(cudaGetLastError());
    *nv = total;
    return GS_OK;
}
