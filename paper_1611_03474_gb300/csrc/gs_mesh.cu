// gs_mesh.cu -- hash-table passes around the triangulation:
//   * conformity for cubes of different sizes (section 2.3: points of the
//     neighbouring cubes inside the current cube are considered): an
//     accepted cube touching, along a face or an edge, a cube at least
//     min_gap levels finer is split into 8 accepted children until no such
//     contact remains (min_gap 2: at most one level between cubes sharing a
//     face or an edge, whose points the constrained vertex values of
//     gs_cons.cu then join; min_gap 1: one size across every shared face and
//     edge);
//   * lattice vertices of the accepted cubes with deterministic ids (owner =
//     smallest (cube, corner) index, then a prefix sum in cube order);
//   * same-size face neighbours of each cube;
//   * welding of the emitted surface points by key (owner = first copy),
//     and remapping of the triangles' keys to vertex ids.
#include "gs_host.cuh"

#include <cmath>
#include <vector>

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
// Each accepted cube F marks every accepted cube C at least min_gap levels
// coarser that contains one of F's 18 face or edge neighbour cells: exactly
// the cubes that touch a cube that much finer along a face or an edge.
__global__ void k_conform_mark(GsHash H, const uint64_t *cubes, int64_t n, int64_t *cnt, int min_gap)
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
        for (int l = lf - min_gap; l >= 0; l--) {
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

// fresh (nullable): 1 for cubes made by this or an earlier split since the
// flags were last cleared (children 1; kept cubes carry their flag over)
__global__ void k_conform_emit(const uint64_t *cubes, int64_t n, const int64_t *off, uint64_t *out,
                               const uint8_t *fresh_in, uint8_t *fresh_out)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= n) return;
    uint64_t k = cubes[i];
    int64_t o = off[i], m = off[i + 1] - off[i];
    if (m == 1) {
        out[o] = k;
        if (fresh_out) fresh_out[o] = fresh_in ? fresh_in[i] : 0;
        return;
    }
    unsigned l = gk_level(k) + 1;
    int64_t x = gk_x(k), y = gk_y(k), z = gk_z(k);
    for (int c = 0; c < 8; c++) {
        out[o + c] = gk_make(2 * x + (c & 1), 2 * y + ((c >> 1) & 1), 2 * z + (c >> 2), GT_CUBE, l);
        if (fresh_out) fresh_out[o + c] = 1;
    }
}

// cnt[i] = 8 splits cube i into its children, 1 keeps it (n + 1 entries,
// scanned in place); in/out: *d_cubes (replaced when any cube splits), *n
int gs_split_counted(uint64_t **d_cubes, int64_t *n, int64_t *cnt, int64_t *splits, cudaStream_t st,
                     uint8_t **d_fresh)
{
    const int64_t m = *n;
    *splits = 0;
    if (m == 0) return GS_OK;
    int64_t *tot = nullptr;
    int rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
    if (rc) return rc;
    cudaMemsetAsync(cnt + m, 0, sizeof(int64_t), st);
    rc = gs_scan_i64(cnt, m + 1, tot, st);
    int64_t total = 0;
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(&total, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = gs_sync(st);
        if (e != cudaSuccess) rc = gs_fail_cuda(e, "split count", __FILE__, __LINE__);
    }
    gs_free(tot, st);
    if (rc || total == m) return rc;
    uint64_t *out = nullptr;
    uint8_t *fr = nullptr;
    rc = gs_alloc((void **)&out, sizeof(uint64_t) * (size_t)total, st);
    if (!rc && d_fresh) rc = gs_alloc((void **)&fr, (size_t)total, st);
    if (rc) { gs_free(out, st); return rc; }
    GS_LAUNCH(k_conform_emit, (unsigned)((m + 255) / 256), 256, 0, st)(*d_cubes, m, cnt, out, d_fresh ? *d_fresh : nullptr,
                                                                       fr);
    gs_free(*d_cubes, st);
    *d_cubes = out;
    if (d_fresh) {
        gs_free(*d_fresh, st);
        *d_fresh = fr;
    }
    *splits = (total - m) / 7;
    *n = total;
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// in/out: *d_cubes (replaced when split), *n
int gs_conformity(uint64_t **d_cubes, int64_t *n, int max_depth, int min_gap, int64_t *splits, unsigned *d_status,
                  cudaStream_t st, uint8_t **d_fresh)
{
    *splits = 0;
    (void)max_depth;
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
        GS_LAUNCH(k_conform_mark, nb, 256, 0, st)(H, *d_cubes, m, cnt, min_gap);
        gs_hash_free(&H, st);
        gs_free(tot, st);
        int64_t ns = 0;
        rc = gs_split_counted(d_cubes, n, cnt, &ns, st, d_fresh);
        gs_free(cnt, st);
        if (rc) return rc;
        if (ns == 0) return GS_OK;
        *splits += ns;
    }
    return gs_fail(GS_ERR_CAPACITY, "conformity did not converge");
}

// ---------------------------------------------------------------- lattice vertices
__device__ __forceinline__ uint64_t corner_key(uint64_t ck, int v, int max_depth)
{
    int64_t s = (int64_t)1 << (max_depth - (int)gk_level(ck));
    return gk_make((gk_x(ck) + (v & 1)) * s, (gk_y(ck) + ((v >> 1) & 1)) * s, (gk_z(ck) + (v >> 2)) * s, GT_VERT, 0);
}

// every corner claims its key's slot (the smallest corner index wins) and
// keeps the slot, so the later passes index the table without probing it.
// A warp holds the corners of 4 consecutive cubes (usually children of one
// octet), many of them shared: lanes with equal keys insert once, through
// their lowest lane, which also has the group's smallest corner index.
__global__ void k_vert_claim(GsHash H, const uint64_t *cubes, int64_t n, int max_depth, int64_t *slot,
                             unsigned *status)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    const bool valid = t < n * 8;
    const unsigned lane = threadIdx.x & 31;
    // corner keys have level 0 (top bits clear): a lane past the end takes a
    // key no corner has, so it matches only itself
    const uint64_t key = valid ? corner_key(cubes[t >> 3], (int)(t & 7), max_depth) : ((1ull << 63) | lane);
    const unsigned grp = __match_any_sync(0xffffffffu, (unsigned long long)key);
    const int leader = __ffs(grp) - 1;
    long long s = -1;
    if (valid && (int)lane == leader) {
        s = gs_hash_insert(H, key, status);
        if (s >= 0) atomicMin((unsigned long long *)&H.vals[s], (unsigned long long)t);
    }
    s = __shfl_sync(0xffffffffu, s, leader);
    if (valid) slot[t] = (int64_t)s;
}

// owner flag per corner (the corner that won its slot)
__global__ void k_vert_owner(GsHash H, int64_t n, int64_t *flag, const int64_t *slot, unsigned *status)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 8) return;
    const int64_t s = slot[t];
    if (s < 0) atomicOr(status, GS_ST_LOOKUP);
    flag[t] = (s >= 0 && H.vals[s] == (uint64_t)t) ? 1 : 0;
}

__global__ void k_vert_write(const uint64_t *cubes, int64_t n, int max_depth, const int64_t *off, const int64_t *slot,
                             uint64_t *vkeys, uint64_t *slot_id)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 8) return;
    if (off[t + 1] == off[t]) return;
    vkeys[off[t]] = corner_key(cubes[t >> 3], (int)(t & 7), max_depth);
    if (slot[t] >= 0) slot_id[slot[t]] = (uint64_t)off[t];
}

__global__ void k_vert_cvid(int64_t n, const int64_t *slot, const uint64_t *slot_id, int32_t *cvid)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 8) return;
    cvid[t] = slot[t] >= 0 ? (int32_t)slot_id[slot[t]] : 0;
}

int gs_lattice_vertices(const uint64_t *d_cubes, int64_t n, int max_depth, uint64_t **d_vkeys, int64_t *nv,
                        int32_t **d_cvid, unsigned *d_status, cudaStream_t st, GsHash *keep_hash,
                        uint64_t **keep_slot_id)
{
    *d_vkeys = nullptr; *d_cvid = nullptr; *nv = 0;
    if (keep_hash) { keep_hash->keys = keep_hash->vals = nullptr; keep_hash->mask = 0; *keep_slot_id = nullptr; }
    if (n <= 0) return GS_OK;
    int64_t m = n * 8;
    GsHash H;
    int rc = gs_hash_make(&H, m / 2 + 8, st);
    if (rc) return rc;
    int64_t *flag = nullptr, *tot = nullptr, *slot = nullptr;
    uint64_t *slot_id = nullptr;
    rc = gs_alloc((void **)&flag, sizeof(int64_t) * (size_t)(m + 1), st);
    if (!rc) rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
    if (!rc) rc = gs_alloc((void **)&slot, sizeof(int64_t) * (size_t)m, st);
    if (!rc) rc = gs_alloc((void **)&slot_id, sizeof(uint64_t) * (size_t)(H.mask + 1), st);
    unsigned nb = (unsigned)((m + 255) / 256);
    if (!rc) {
        GS_LAUNCH(k_vert_claim, nb, 256, 0, st)(H, d_cubes, n, max_depth, slot, d_status);
        cudaMemsetAsync(flag + m, 0, sizeof(int64_t), st);
        GS_LAUNCH(k_vert_owner, nb, 256, 0, st)(H, n, flag, slot, d_status);
        rc = gs_scan_i64(flag, m + 1, tot, st);
    }
    int64_t total = 0;
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(&total, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = gs_sync(st);
        if (e != cudaSuccess) rc = gs_fail_cuda(e, "vertex count", __FILE__, __LINE__);
    }
    if (!rc) rc = gs_alloc((void **)d_vkeys, sizeof(uint64_t) * (size_t)(total + 1), st);
    if (!rc) rc = gs_alloc((void **)d_cvid, sizeof(int32_t) * (size_t)m, st);
    if (!rc) {
        // unused slots keep the sentinel ~0 (gs_lattice_extend tells new keys by it)
        if (keep_hash) cudaMemsetAsync(slot_id, 0xFF, sizeof(uint64_t) * (size_t)(H.mask + 1), st);
        GS_LAUNCH(k_vert_write, nb, 256, 0, st)(d_cubes, n, max_depth, flag, slot, *d_vkeys, slot_id);
        GS_LAUNCH(k_vert_cvid, nb, 256, 0, st)(n, slot, slot_id, *d_cvid);
    }
    gs_free(flag, st); gs_free(tot, st); gs_free(slot, st);
    if (!rc && keep_hash) {
        // key -> slot stays; slot -> vertex id through slot_id
        *keep_hash = H;
        *keep_slot_id = slot_id;
    } else {
        gs_free(slot_id, st);
        gs_hash_free(&H, st);
    }
    if (rc) { gs_free(*d_vkeys, st); gs_free(*d_cvid, st); *d_vkeys = nullptr; *d_cvid = nullptr; return rc; }
    GS_CHECK(cudaGetLastError());
    *nv = total;
    return GS_OK;
}

// ---------------------------------------------------------------- growing the lattice
// After splits the vertex set only grows (a split cube's corners are corners
// of its children).  gs_lattice_extend keeps the previous lattice's vertex
// ids, appends the corners of the fresh cubes that it lacked (in the order
// of first appearance among the fresh cubes' corners) and rebuilds the
// corner ids of every cube by hash lookups.
__global__ void k_fresh_flags(const uint8_t *__restrict__ fresh, int64_t n, int64_t *__restrict__ flag)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n) flag[i] = fresh[i] ? 1 : 0;
}
__global__ void k_fresh_list(const int64_t *__restrict__ off, int64_t n, int64_t *__restrict__ list)
{
    const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i < n && off[i + 1] != off[i]) list[off[i]] = i;
}
// corner t of fresh cube list[t >> 3]: insert its key; vals elects the
// smallest t among the corners claiming a slot
__global__ void k_vert_claim_list(GsHash H, const uint64_t *__restrict__ cubes, const int64_t *__restrict__ list,
                                  int64_t m, int max_depth, int64_t *__restrict__ slot, unsigned *status)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * 8) return;
    const uint64_t key = corner_key(cubes[list[t >> 3]], (int)(t & 7), max_depth);
    const int64_t s = gs_hash_insert(H, key, status);
    if (s >= 0) atomicMin((unsigned long long *)&H.vals[s], (unsigned long long)t);
    slot[t] = s;
}
// a corner owns a new vertex when its slot had no id and it won the slot
__global__ void k_vert_owner_new(GsHash H, int64_t m, const int64_t *__restrict__ slot,
                                 const uint64_t *__restrict__ slot_id, int64_t *__restrict__ flag, unsigned *status)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * 8) return;
    const int64_t s = slot[t];
    if (s < 0) atomicOr(status, GS_ST_LOOKUP);
    flag[t] = (s >= 0 && slot_id[s] == ~0ull && H.vals[s] == (uint64_t)t) ? 1 : 0;
}
__global__ void k_vert_write_new(const uint64_t *__restrict__ cubes, const int64_t *__restrict__ list, int64_t m,
                                 int max_depth, const int64_t *__restrict__ off, const int64_t *__restrict__ slot,
                                 int64_t base, uint64_t *__restrict__ vkeys, uint64_t *__restrict__ slot_id)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= m * 8 || off[t + 1] == off[t]) return;
    vkeys[base + off[t]] = corner_key(cubes[list[t >> 3]], (int)(t & 7), max_depth);
    slot_id[slot[t]] = (uint64_t)(base + off[t]);
}
__global__ void k_vert_cvid_find(GsHash H, const uint64_t *__restrict__ slot_id, const uint64_t *__restrict__ cubes,
                                 int64_t n, int max_depth, int32_t *__restrict__ cvid, unsigned *status)
{
    const int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n * 8) return;
    const int64_t s = gs_hash_find(H, corner_key(cubes[t >> 3], (int)(t & 7), max_depth));
    uint64_t id = s >= 0 ? slot_id[s] : ~0ull;
    if (id == ~0ull) {
        atomicOr(status, GS_ST_LOOKUP);
        id = 0;
    }
    cvid[t] = (int32_t)id;
}

int gs_lattice_extend(const uint64_t *d_cubes, int64_t n, const uint8_t *d_fresh, int max_depth, const GsHash &H,
                      uint64_t *d_slot_id, uint64_t **d_vkeys, int64_t *nv, int32_t **d_cvid, int64_t *n_added,
                      unsigned *d_status, cudaStream_t st)
{
    *n_added = 0;
    int64_t *flag = nullptr, *tot = nullptr, *list = nullptr, *slot = nullptr;
    uint64_t *vk = nullptr;
    int32_t *cv = nullptr;
    auto host_count = [&](int64_t *out) {
        cudaError_t e = cudaMemcpyAsync(out, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = gs_sync(st);
        return e == cudaSuccess ? GS_OK : gs_fail_cuda(e, "lattice extension", __FILE__, __LINE__);
    };
    int rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
    if (!rc) rc = gs_alloc((void **)&flag, sizeof(int64_t) * (size_t)(n + 1), st);
    int64_t m = 0;
    if (!rc) {
        cudaMemsetAsync(flag + n, 0, sizeof(int64_t), st);
        GS_LAUNCH(k_fresh_flags, (unsigned)((n + 255) / 256), 256, 0, st)(d_fresh, n, flag);
        rc = gs_scan_i64(flag, n + 1, tot, st);
    }
    if (!rc) rc = host_count(&m);
    if (!rc && m > 0) rc = gs_alloc((void **)&list, sizeof(int64_t) * (size_t)m, st);
    if (!rc && m > 0) GS_LAUNCH(k_fresh_list, (unsigned)((n + 255) / 256), 256, 0, st)(flag, n, list);
    gs_free(flag, st);
    flag = nullptr;
    int64_t added = 0;
    if (!rc && m > 0) {
        const int64_t c8 = m * 8;
        const unsigned nb = (unsigned)((c8 + 255) / 256);
        rc = gs_alloc((void **)&slot, sizeof(int64_t) * (size_t)c8, st);
        if (!rc) rc = gs_alloc((void **)&flag, sizeof(int64_t) * (size_t)(c8 + 1), st);
        if (!rc) {
            GS_LAUNCH(k_vert_claim_list, nb, 256, 0, st)(H, d_cubes, list, m, max_depth, slot, d_status);
            cudaMemsetAsync(flag + c8, 0, sizeof(int64_t), st);
            GS_LAUNCH(k_vert_owner_new, nb, 256, 0, st)(H, m, slot, d_slot_id, flag, d_status);
            rc = gs_scan_i64(flag, c8 + 1, tot, st);
        }
        if (!rc) rc = host_count(&added);
        if (!rc) rc = gs_alloc((void **)&vk, sizeof(uint64_t) * (size_t)(*nv + added + 1), st);
        if (!rc) {
            GS_CHECK(cudaMemcpyAsync(vk, *d_vkeys, sizeof(uint64_t) * (size_t)*nv, cudaMemcpyDeviceToDevice, st));
            if (added > 0)
                GS_LAUNCH(k_vert_write_new, nb, 256, 0, st)(d_cubes, list, m, max_depth, flag, slot, *nv, vk,
                                                            d_slot_id);
        }
    }
    if (!rc) rc = gs_alloc((void **)&cv, sizeof(int32_t) * (size_t)(n * 8), st);
    if (!rc)
        GS_LAUNCH(k_vert_cvid_find, (unsigned)((n * 8 + 255) / 256), 256, 0, st)(H, d_slot_id, d_cubes, n, max_depth,
                                                                                 cv, d_status);
    gs_free(tot, st); gs_free(flag, st); gs_free(list, st); gs_free(slot, st);
    if (rc) { gs_free(vk, st); gs_free(cv, st); return rc; }
    GS_CHECK(cudaGetLastError());
    if (vk) {
        gs_free(*d_vkeys, st);
        *d_vkeys = vk;
    }
    gs_free(*d_cvid, st);
    *d_cvid = cv;
    *nv += added;
    *n_added = added;
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

int gs_neighbours(const uint64_t *d_cubes, int64_t n, int32_t **d_nbr, unsigned *d_status, cudaStream_t st,
                  GsHash *keep_hash)
{
    *d_nbr = nullptr;
    if (keep_hash) { keep_hash->keys = keep_hash->vals = nullptr; keep_hash->mask = 0; }
    if (n <= 0) return GS_OK;
    GsHash H;
    int rc = gs_hash_make(&H, n, st);
    if (rc) return rc;
    GS_LAUNCH(k_hash_index, (unsigned)((n + 255) / 256), 256, 0, st)(H, d_cubes, n, d_status);
    rc = gs_alloc((void **)d_nbr, sizeof(int32_t) * 6 * (size_t)n, st);
    if (!rc) GS_LAUNCH(k_neighbours, (unsigned)((6 * n + 255) / 256), 256, 0, st)(H, d_cubes, n, *d_nbr);
    if (!rc && keep_hash) *keep_hash = H;
    else gs_hash_free(&H, st);
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}

// ---------------------------------------------------------------- weld
// every point claims its key's slot (the smallest point index wins) and
// keeps the slot for the owner and write passes
__global__ void k_weld_claim(GsHash H, const uint64_t *pk, int64_t n, int64_t *slot, unsigned *status)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    int64_t s = gs_hash_insert(H, pk[t], status);
    slot[t] = s;
    if (s >= 0) atomicMin((unsigned long long *)&H.vals[s], (unsigned long long)t);
}
__global__ void k_weld_owner(GsHash H, int64_t n, int64_t *flag, const int64_t *slot)
{
    int64_t t = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const int64_t s = slot[t];
    flag[t] = (s >= 0 && H.vals[s] == (uint64_t)t) ? 1 : 0;
}
__global__ void k_weld_write(const uint64_t *pk, const double *pxyz, int64_t n, const int64_t *off, const int64_t *slot,
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
    if (slot[t] >= 0) slot_id[slot[t]] = (uint64_t)id;
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
    int64_t *flag = nullptr, *tot = nullptr, *slot = nullptr;
    uint64_t *slot_id = nullptr;
    rc = gs_alloc((void **)&flag, sizeof(int64_t) * (size_t)(npt + 1), st);
    if (!rc) rc = gs_alloc((void **)&tot, sizeof(int64_t), st);
    if (!rc) rc = gs_alloc((void **)&slot, sizeof(int64_t) * (size_t)npt, st);
    if (!rc) rc = gs_alloc((void **)&slot_id, sizeof(uint64_t) * (size_t)(H.mask + 1), st);
    unsigned nb = (unsigned)((npt + 255) / 256);
    if (!rc) {
        GS_LAUNCH(k_weld_claim, nb, 256, 0, st)(H, d_pk, npt, slot, d_status);
        cudaMemsetAsync(flag + npt, 0, sizeof(int64_t), st);
        GS_LAUNCH(k_weld_owner, nb, 256, 0, st)(H, npt, flag, slot);
        rc = gs_scan_i64(flag, npt + 1, tot, st);
    }
    int64_t total = 0;
    if (!rc) {
        cudaError_t e = cudaMemcpyAsync(&total, tot, sizeof(int64_t), cudaMemcpyDeviceToHost, st);
        if (e == cudaSuccess) e = gs_sync(st);
        if (e != cudaSuccess) rc = gs_fail_cuda(e, "weld count", __FILE__, __LINE__);
    }
    if (!rc) rc = gs_alloc((void **)d_vkeys, sizeof(uint64_t) * (size_t)(total + 1), st);
    if (!rc) rc = gs_alloc((void **)d_vxyz, sizeof(double) * 3 * (size_t)(total + 1), st);
    if (!rc) rc = gs_alloc((void **)d_tri, sizeof(int32_t) * 3 * (size_t)(ntri + 1), st);
    if (!rc) {
        GS_LAUNCH(k_weld_write, nb, 256, 0, st)(d_pk, d_pxyz, npt, flag, slot, *d_vkeys, *d_vxyz, slot_id);
        if (ntri > 0)
            GS_LAUNCH(k_weld_tris, (unsigned)((3 * ntri + 255) / 256), 256, 0, st)(H, slot_id, d_tk, ntri, *d_tri, d_status);
    }
    gs_free(slot, st); gs_free(flag, st); gs_free(tot, st); gs_free(slot_id, st);
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

// ---------------------------------------------------------------- mesh check
// Pairs of triangles that share no vertex and intersect (the paper reports
// none for its meshes).  Triangles are binned by their centroid on a grid
// whose cell is at least the largest triangle extent, so any intersecting
// pair lies in the same or in neighbouring cells; each pair is tested once
// (by its lower index) with the separating-axis test on the 11 candidate
// axes (2 normals, 9 edge cross products), FP64, counting only pairs with no
// separating gap larger than tol.
__global__ void k_tri_bins(const double *v, const int32_t *t, int64_t nt, const double *lo, double inv, const int *dims,
                           int32_t *cell)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= nt) return;
    int cc[3];
    for (int a = 0; a < 3; a++) {
        double m = (v[3 * (int64_t)t[3 * i] + a] + v[3 * (int64_t)t[3 * i + 1] + a] + v[3 * (int64_t)t[3 * i + 2] + a]) / 3.0;
        int k = (int)floor((m - lo[a]) * inv);
        cc[a] = k < 0 ? 0 : (k >= dims[a] ? dims[a] - 1 : k);
    }
    cell[i] = cc[0] + dims[0] * (cc[1] + dims[1] * cc[2]);
}

__device__ __forceinline__ void tri_project(const double (*p)[3], const double *ax, double &mn, double &mx)
{
    double d0 = p[0][0] * ax[0] + p[0][1] * ax[1] + p[0][2] * ax[2];
    double d1 = p[1][0] * ax[0] + p[1][1] * ax[1] + p[1][2] * ax[2];
    double d2 = p[2][0] * ax[0] + p[2][1] * ax[1] + p[2][2] * ax[2];
    mn = fmin(d0, fmin(d1, d2));
    mx = fmax(d0, fmax(d1, d2));
}

// true when the triangles overlap by more than tol along every candidate
// separating axis (a separating gap, or an overlap of at most tol, on any
// axis means no intersection)
__device__ bool tris_intersect(const double (*P)[3], const double (*Q)[3], double tol)
{
    double eP[3][3], eQ[3][3];
    for (int k = 0; k < 3; k++)
        for (int a = 0; a < 3; a++) {
            eP[k][a] = P[(k + 1) % 3][a] - P[k][a];
            eQ[k][a] = Q[(k + 1) % 3][a] - Q[k][a];
        }
    auto cross = [](const double *x, const double *y, double *o) {
        o[0] = x[1] * y[2] - x[2] * y[1];
        o[1] = x[2] * y[0] - x[0] * y[2];
        o[2] = x[0] * y[1] - x[1] * y[0];
    };
    auto separated = [&](const double *axis) {
        double n2 = axis[0] * axis[0] + axis[1] * axis[1] + axis[2] * axis[2];
        if (n2 <= 1e-30) return false;   // degenerate axis
        double inv = 1.0 / sqrt(n2), ax[3] = {axis[0] * inv, axis[1] * inv, axis[2] * inv};
        double a0, a1, b0, b1;
        tri_project(P, ax, a0, a1);
        tri_project(Q, ax, b0, b1);
        return a1 <= b0 + tol || b1 <= a0 + tol;
    };
    double nP[3], nQ[3];
    cross(eP[0], eP[1], nP);
    cross(eQ[0], eQ[1], nQ);
    double lP = sqrt(nP[0] * nP[0] + nP[1] * nP[1] + nP[2] * nP[2]);
    bool coplanar = lP > 0.0;
    for (int k = 0; k < 3 && coplanar; k++) {
        double d = (nP[0] * (Q[k][0] - P[0][0]) + nP[1] * (Q[k][1] - P[0][1]) + nP[2] * (Q[k][2] - P[0][2])) / lP;
        coplanar = fabs(d) <= tol;
    }
    if (coplanar) {
        // in the common plane: the in-plane normals of the six edges
        for (int s = 0; s < 2; s++)
            for (int k = 0; k < 3; k++) {
                double ax[3];
                cross(s ? eQ[k] : eP[k], nP, ax);
                if (separated(ax)) return false;
            }
        return true;
    }
    if (separated(nP) || separated(nQ)) return false;
    for (int i = 0; i < 3; i++)
        for (int j = 0; j < 3; j++) {
            double ax[3];
            cross(eP[i], eQ[j], ax);
            if (separated(ax)) return false;
        }
    return true;
}

__global__ void k_tri_pairs(const double *v, const int32_t *t, int64_t nt, const int32_t *order,
                            const int32_t *cell_start, const int32_t *cell, const int *dims, double tol,
                            unsigned long long *count)
{
    int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    unsigned long long found = 0;
    if (i < nt) {
        int32_t ti[3] = {t[3 * i], t[3 * i + 1], t[3 * i + 2]};
        double P[3][3];
        for (int k = 0; k < 3; k++)
            for (int a = 0; a < 3; a++) P[k][a] = v[3 * (int64_t)ti[k] + a];
        int c = cell[i];
        int cx = c % dims[0], cy = (c / dims[0]) % dims[1], cz = c / (dims[0] * dims[1]);
        for (int dz = -1; dz <= 1; dz++)
            for (int dy = -1; dy <= 1; dy++)
                for (int dx = -1; dx <= 1; dx++) {
                    int x = cx + dx, y = cy + dy, z = cz + dz;
                    if (x < 0 || y < 0 || z < 0 || x >= dims[0] || y >= dims[1] || z >= dims[2]) continue;
                    int nc = x + dims[0] * (y + dims[1] * z);
                    for (int s = cell_start[nc]; s < cell_start[nc + 1]; s++) {
                        int64_t j = order[s];
                        if (j <= i) continue;
                        int32_t tj[3] = {t[3 * j], t[3 * j + 1], t[3 * j + 2]};
                        bool shared = false;
                        for (int a = 0; a < 3; a++)
                            for (int b = 0; b < 3; b++) shared |= ti[a] == tj[b];
                        if (shared) continue;
                        double Q[3][3];
                        for (int k = 0; k < 3; k++)
                            for (int a = 0; a < 3; a++) Q[k][a] = v[3 * (int64_t)tj[k] + a];
                        if (tris_intersect(P, Q, tol)) found++;
                    }
                }
    }
    for (int o = 16; o > 0; o >>= 1) found += __shfl_xor_sync(0xffffffffu, found, o);
    if ((threadIdx.x & 31) == 0 && found) atomicAdd(count, found);
}

int gs_count_intersections(const double *d_v, int64_t nv, const int32_t *d_t, int64_t nt, double tol,
                           int64_t *n_pairs, cudaStream_t st)
{
    *n_pairs = 0;
    if (nt <= 1) return GS_OK;
    // bounding box and largest triangle extent on the host (one pass over a
    // copy would do; the vertices are read back once here for simplicity)
    std::vector<double> hv((size_t)nv * 3);
    std::vector<int32_t> ht((size_t)nt * 3);
    GS_CHECK(cudaMemcpyAsync(hv.data(), d_v, sizeof(double) * hv.size(), cudaMemcpyDeviceToHost, st));
    GS_CHECK(cudaMemcpyAsync(ht.data(), d_t, sizeof(int32_t) * ht.size(), cudaMemcpyDeviceToHost, st));
    GS_CHECK(gs_sync(st));
    double lo[3] = {1e300, 1e300, 1e300}, hi[3] = {-1e300, -1e300, -1e300}, ext = 0.0;
    for (int64_t i = 0; i < nv; i++)
        for (int a = 0; a < 3; a++) { lo[a] = fmin(lo[a], hv[3 * i + a]); hi[a] = fmax(hi[a], hv[3 * i + a]); }
    for (int64_t i = 0; i < nt; i++)
        for (int a = 0; a < 3; a++) {
            double x0 = hv[3 * (int64_t)ht[3 * i] + a], x1 = hv[3 * (int64_t)ht[3 * i + 1] + a],
                   x2 = hv[3 * (int64_t)ht[3 * i + 2] + a];
            ext = fmax(ext, fmax(x0, fmax(x1, x2)) - fmin(x0, fmin(x1, x2)));
        }
    // two intersecting triangles of extent <= ext have centroids within 4/3 ext
    // per axis, so a cell of that size puts them in the same or adjacent cells;
    // larger cells when that would exceed ~4 cells per triangle
    double cellsz = fmax(4.0 / 3.0 * ext * (1.0 + 1e-9), 1e-6);
    double vol = 1.0;
    for (int a = 0; a < 3; a++) vol *= fmax(hi[a] - lo[a], cellsz);
    cellsz = fmax(cellsz, cbrt(vol / (4.0 * (double)nt)));
    int dims[3];
    for (int a = 0; a < 3; a++) dims[a] = (int)((int64_t)floor((hi[a] - lo[a]) / cellsz) + 1);
    const int64_t ncell = (int64_t)dims[0] * dims[1] * dims[2];
    double *d_lo = nullptr;
    int *d_dims = nullptr;
    int32_t *cell = nullptr, *order = nullptr, *start = nullptr;
    unsigned long long *cnt = nullptr;
    int rc = gs_alloc((void **)&d_lo, 3 * sizeof(double), st);
    if (!rc) rc = gs_alloc((void **)&d_dims, 3 * sizeof(int), st);
    if (!rc) rc = gs_alloc((void **)&cell, sizeof(int32_t) * (size_t)nt, st);
    if (!rc) rc = gs_alloc((void **)&cnt, sizeof(unsigned long long), st);
    if (rc) { gs_free(d_lo, st); gs_free(d_dims, st); gs_free(cell, st); gs_free(cnt, st); return rc; }
    GS_CHECK(cudaMemcpyAsync(d_lo, lo, 3 * sizeof(double), cudaMemcpyHostToDevice, st));
    GS_CHECK(cudaMemcpyAsync(d_dims, dims, 3 * sizeof(int), cudaMemcpyHostToDevice, st));
    GS_LAUNCH(k_tri_bins, (unsigned)((nt + 255) / 256), 256, 0, st)(d_v, d_t, nt, d_lo, 1.0 / cellsz, d_dims, cell);
    // counting sort of the triangles by cell on the host (cell array read back)
    std::vector<int32_t> hc((size_t)nt), hs((size_t)ncell + 1, 0), ho((size_t)nt);
    GS_CHECK(cudaMemcpyAsync(hc.data(), cell, sizeof(int32_t) * (size_t)nt, cudaMemcpyDeviceToHost, st));
    GS_CHECK(gs_sync(st));
    for (int64_t i = 0; i < nt; i++) hs[(size_t)hc[i] + 1]++;
    for (int64_t k = 0; k < ncell; k++) hs[(size_t)k + 1] += hs[(size_t)k];
    {
        std::vector<int32_t> fill(hs.begin(), hs.end() - 1);
        for (int64_t i = 0; i < nt; i++) ho[(size_t)fill[(size_t)hc[i]]++] = (int32_t)i;
    }
    rc = gs_alloc((void **)&order, sizeof(int32_t) * (size_t)nt, st);
    if (!rc) rc = gs_alloc((void **)&start, sizeof(int32_t) * (size_t)(ncell + 1), st);
    if (!rc) {
        GS_CHECK(cudaMemcpyAsync(order, ho.data(), sizeof(int32_t) * (size_t)nt, cudaMemcpyHostToDevice, st));
        GS_CHECK(cudaMemcpyAsync(start, hs.data(), sizeof(int32_t) * (size_t)(ncell + 1), cudaMemcpyHostToDevice, st));
        GS_CHECK(cudaMemsetAsync(cnt, 0, sizeof(unsigned long long), st));
        GS_LAUNCH(k_tri_pairs, (unsigned)((nt + 127) / 128), 128, 0, st)(d_v, d_t, nt, order, start, cell, d_dims, tol,
                                                                         cnt);
        unsigned long long h = 0;
        GS_CHECK(cudaMemcpyAsync(&h, cnt, sizeof(h), cudaMemcpyDeviceToHost, st));
        GS_CHECK(gs_sync(st));
        *n_pairs = (int64_t)h;
    }
    gs_free(d_lo, st); gs_free(d_dims, st); gs_free(cell, st); gs_free(cnt, st); gs_free(order, st); gs_free(start, st);
    if (rc) return rc;
    GS_CHECK(cudaGetLastError());
    return GS_OK;
}
