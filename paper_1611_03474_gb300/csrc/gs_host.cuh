// gs_host.cuh -- host-side interfaces between the library's translation units.
#pragma once
#include "gs_internal.cuh"

#include <functional>

// gs_guard.cu: host waits with a deadline (cudaErrorTimeout after it) and
// host-side fault injection (environment GS_FAULT); gs_guard_begin at each
// API call
cudaError_t gs_sync(cudaStream_t st);
void gs_guard_begin(void);
bool gs_fault_alloc(void);
bool gs_fault_capacity(int level);

struct GsAtomsSoA {
    double *x, *y, *z, *r, *R2, *w;
    float *fx, *fy, *fz;
    float *hx, *lx, *hy, *ly, *hz, *lz, *fw, *fR2, *fr2, *lr2;
};

// gs_bin.cu
int gs_prep_atoms(const double *d_xyz, const double *d_r, int64_t n, double D, double KD, double *d_R2, double *d_w,
                  double bbox[6], double *r2max, unsigned *d_status, cudaStream_t st);
// stable permutation sorting int32 keys in [0, nkeys) (d_keys is clobbered)
int gs_sort_perm(int32_t *d_keys, int64_t n, int64_t nkeys, int32_t *d_perm, cudaStream_t st);
int gs_build_cells(const double *d_xyz, int64_t n, const double origin[3], double cell, const int cdim[3],
                   int32_t *d_cell_start, int32_t *d_perm, cudaStream_t st);
int gs_gather_atoms(const int32_t *d_perm, int64_t n, const double *d_xyz, const double *d_r, const double *d_R2,
                    const double *d_w, const double origin[3], double cell, const int cdim[3], GsAtomsSoA *soa,
                    cudaStream_t st);

// gs_level.cu
int gs_quadrature_init(void);
// accumulate A for the 8 children of each parent (level-1 coords in parents,
// or the implicit root blocks when parents == NULL); vmask (nullable) selects
// children; A_out [n_oct*8][64]
// d_probs, d_mol (nullable, the batched form): octet o belongs to molecule
// d_mol[o] whose problem is d_probs[d_mol[o]] (P then only supplies what the
// molecules share: D, c, precision, the lattice spacing)
int gs_accum_f64(const GsProblem &P, int level, const uint64_t *d_parents, const uint8_t *d_vmask, int64_t n_oct,
                 double *d_A, unsigned long long *d_pairs, unsigned *d_status, cudaStream_t st, float *ms = nullptr,
                 const GsProblem *d_probs = nullptr, const int32_t *d_mol = nullptr);
int gs_estimate_f64(const GsProblem &P, int level, const double *d_A, int64_t n_cubes, const uint64_t *d_parents,
                    const uint8_t *d_vmask, uint8_t *d_dec, double *d_bounds, cudaStream_t st);
// mixed precision: FP32 accumulate (Kahan) + error bound, FP32 estimate with margins
int gs_accum_f32(const GsProblem &P, int level, const uint64_t *d_parents, const uint8_t *d_vmask, int64_t n_oct,
                 float *d_A, float *d_err, unsigned long long *d_pairs, unsigned *d_status, cudaStream_t st,
                 float *ms = nullptr, unsigned long long *d_atom_octets = nullptr, const GsProblem *d_probs = nullptr,
                 const int32_t *d_mol = nullptr);
int gs_estimate_f32(const GsProblem &P, int level, const float *d_A, const float *d_err, int64_t n_cubes,
                    const uint64_t *d_parents, const uint8_t *d_vmask, uint8_t *d_dec, uint8_t *d_flag,
                    cudaStream_t st, unsigned long long *d_why = nullptr, float *d_dbg = nullptr);

// gs_field.cu
int gs_field_f64(const GsProblem &P, const uint64_t *d_vkeys, const double *d_points, int64_t n, double *d_phi,
                 double *d_grad, unsigned long long *d_terms, cudaStream_t st);
// d_mark (n + 1 entries, consumed): the marked vertices re-evaluated in
// double-word FP32 (value and bound), and those whose sign relative to c is
// still within 4 bounds in FP64 (bound 0); *n_dw, *n_fp64 of them
int gs_field_refine(const GsProblem &P, const uint64_t *d_vkeys, int64_t n, int64_t *d_mark, double *d_phi,
                    float *d_err, int64_t *n_dw, int64_t *n_fp64, cudaStream_t st);
// phi and its bound at lattice vertices (d_vkeys) or points, double-word FP32
int gs_field_dw(const GsProblem &P, const uint64_t *d_vkeys, const double *d_points, int64_t n, double *d_phi,
                float *d_err, unsigned long long *d_terms, cudaStream_t st);
int gs_field_init(void);
// re-evaluate in FP64 the vertices with mark[v] = 1 (mark: n + 1 entries, scanned in place)
int gs_field_recompute(const GsProblem &P, const uint64_t *d_vkeys, int64_t n, int64_t *d_mark, double *d_phi,
                       float *d_err, int64_t *n_recomputed, cudaStream_t st);
// mark[v] = 1 where |phi - c| is within 4 bounds
int gs_field_flag_near(const GsProblem &P, const double *d_phi, const float *d_err, int64_t n, int64_t *d_mark,
                       cudaStream_t st);
int gs_field_f32(const GsProblem &P, const uint64_t *d_vkeys, const double *d_points, int64_t n, double *d_phi,
                 double *d_grad, float *d_err, unsigned long long *d_terms, cudaStream_t st);
// d_A / d_nextA (optional): the level's tensors in, the split cubes' tensors
// out in the order of the next level's parents (for re-expansion)
int gs_level_compact(const GsProblem &P, int level, const uint64_t *d_parents, const uint8_t *d_vmask, int64_t n_oct,
                     const uint8_t *d_dec, uint64_t **d_next, int64_t *n_next, uint64_t *d_acc_base,
                     int64_t acc_cap, int64_t *n_acc, unsigned long long *d_counters, cudaStream_t st,
                     const double *d_A = nullptr, double **d_nextA = nullptr, const int32_t *d_mol = nullptr,
                     int32_t **d_next_mol = nullptr, int32_t *d_acc_mol = nullptr);
// child tensors [n_oct][8][64] re-expanded from the parents' tensors [n_oct][64]
int gs_reexpand(const double *d_Apar, int64_t n_oct, double *d_A, cudaStream_t st);

int gs_level_mixed(const GsProblem &P, int level, const uint64_t *d_parents, int64_t n_oct, uint8_t *d_dec,
                   unsigned long long *d_pairs, unsigned long long *d_rechecked, unsigned long long *d_mism,
                   bool both, unsigned *d_status, cudaStream_t st, float *ms = nullptr,
                   unsigned long long *d_why = nullptr, const GsProblem *d_probs = nullptr,
                   const int32_t *d_mol = nullptr, const uint8_t *d_vmask = nullptr);
int gs_root_blocks(const GsProblem &P, uint64_t **d_keys, int64_t *n, cudaStream_t st);
// batched form: the root blocks of G molecules (probs: host records) with
// their valid-child masks and molecule indices; per-molecule decision counts
// (d_cnt [G][5], accumulated); accepted cubes of one compaction part to
// their molecules' arrays (outs[g][j + q0 + shift[g]], g = mol[j])
int gs_root_blocks_batch(const GsProblem *probs, int G, uint64_t **d_keys, uint8_t **d_vmask, int32_t **d_mol,
                         int64_t *n, cudaStream_t st);
int gs_level_count_mol(const uint8_t *d_dec, int64_t n_cubes, const int32_t *d_mol, unsigned long long *d_cnt,
                       cudaStream_t st);
int gs_scatter_cubes(const uint64_t *d_acc, const int32_t *d_acc_mol, int64_t n, int64_t q0, const int64_t *d_shift,
                     uint64_t *const *d_outs, const int64_t *d_cap, unsigned *d_status, cudaStream_t st);

// gs_mesh.cu
int gs_hash_make(GsHash *H, int64_t n, cudaStream_t st);
void gs_hash_free(GsHash *H, cudaStream_t st);
// min_gap: split a cube that touches one at least this many levels finer
int gs_conformity(uint64_t **d_cubes, int64_t *n, int max_depth, int min_gap, int64_t *splits, unsigned *d_status,
                  cudaStream_t st, uint8_t **d_fresh = nullptr);
int gs_split_counted(uint64_t **d_cubes, int64_t *n, int64_t *cnt, int64_t *splits, cudaStream_t st,
                     uint8_t **d_fresh = nullptr);
// lattice of a cube list grown by splits (fresh[ci] = 1 for the new cubes):
// the previous vertices keep their ids, the new ones are appended; *d_vkeys
// and *d_cvid are replaced (the old arrays freed), H and d_slot_id extended
int gs_lattice_extend(const uint64_t *d_cubes, int64_t n, const uint8_t *d_fresh, int max_depth, const GsHash &H,
                      uint64_t *d_slot_id, uint64_t **d_vkeys, int64_t *nv, int32_t **d_cvid, int64_t *n_added,
                      unsigned *d_status, cudaStream_t st);
// keep_hash (nullable): the key -> slot table of the vertices is handed over
// (free with gs_hash_free), with *keep_slot_id mapping a slot to the vertex id
int gs_lattice_vertices(const uint64_t *d_cubes, int64_t n, int max_depth, uint64_t **d_vkeys, int64_t *nv,
                        int32_t **d_cvid, unsigned *d_status, cudaStream_t st, GsHash *keep_hash = nullptr,
                        uint64_t **keep_slot_id = nullptr);
// keep_hash (nullable): the cube key -> index table is handed over
int gs_neighbours(const uint64_t *d_cubes, int64_t n, int32_t **d_nbr, unsigned *d_status, cudaStream_t st,
                  GsHash *keep_hash = nullptr);
int gs_weld(const uint64_t *d_pk, const double *d_pxyz, int64_t npt, const uint64_t *d_tk, int64_t ntri,
            uint64_t **d_vkeys, double **d_vxyz, int64_t *nv, int32_t **d_tri, unsigned *d_status, cudaStream_t st);

// gs_cons.cu: constrained vertex values for cubes of different sizes
struct GsCons {
    int8_t *lev;     // [nv] level of the constraining face or edge, -1 free
    int32_t *src;    // [nv][4] source vertex ids (-1 unused)
    double *t;       // [nv][2] fractions along the edge, or along the face's axes
    int64_t nv;
    int64_t ncons;   // constrained vertices (after gs_cons_find)
    int32_t *list;   // [ncons] the constrained vertices grouped by level (after gs_cons_find)
    int64_t loff[22];   // level l's group: list[loff[l] .. loff[l + 1])
};
int gs_cons_alloc(GsCons *K, int64_t nv, cudaStream_t st);
void gs_cons_free(GsCons *K, cudaStream_t st);
// d_mark (nullable): marks every constrained vertex and its sources;
// d_scratch: one device counter
int gs_cons_find(GsCons *K, const GsHash &hc, const GsHash &hv, const uint64_t *d_slot_id, const uint64_t *d_vkeys,
                 int md, int64_t *d_mark, unsigned long long *d_scratch, unsigned *d_status, cudaStream_t st);
// replaces the constrained values in d_phi (coarse to fine); d_err
// (nullable) carries the FP32 bounds through the interpolants; d_mark
// (nullable) marks the sources of values within 4 bounds of c; with d_split
// (n + 1 entries per cube, preset to 1) counts the sign disagreements with
// the vertices' own field values and sets 8 for the cubes to split
int gs_cons_apply(const GsCons &K, const GsHash &hc, const uint64_t *d_vkeys, int md, double c, double *d_phi,
                  float *d_err, int64_t *d_mark, int64_t *d_split, int64_t *n_flip, unsigned long long *d_scratch,
                  cudaStream_t st);
// marks on constrained vertices pass to their sources, fine to coarse
int gs_cons_mark_up(const GsCons &K, int md, int64_t *d_mark, cudaStream_t st);

int gs_mixed_flags(const GsCons &K, const uint64_t *d_cubes, int64_t n, const int32_t *d_cvid, const GsHash &hv,
                   const uint64_t *d_slot_id, int md, uint8_t *d_mixed, int64_t *n_mixed,
                   unsigned long long *d_scratch, cudaStream_t st);
int gs_cons_unmark(const GsCons &K, int64_t *d_mark, cudaStream_t st);
int gs_cons_adjoint(const GsCons &K, int md, double *d_lambda, cudaStream_t st);
int gs_fill_i64(int64_t *d_a, int64_t n, int64_t v, cudaStream_t st);

// gs_tri.cu
struct TriCtx {
    const uint64_t *cubes;
    const int32_t *cvid;    // [ncubes][8] lattice-vertex ids of the corners
    const int32_t *nbr;     // [ncubes][6]: same-size neighbour across face (axis a, side s) at 2a+s, -1 if none
    const double *phi;      // field at lattice vertices
    int64_t ncubes;
    double c;
    double origin[3];
    double min_edge;
    int max_depth;
    // fold roots per cube, filled by gs_triangulate before the tracing passes:
    // fcount[4 ci + a] roots of axis a at froot[12 ci + 4 a + 2 r + (0: u, 1: v)]
    const uint8_t *fcount = nullptr;
    const double *froot = nullptr;
    // cubes of different sizes: per-cube flag of a mixed-size contact (null:
    // all cubes that share a face or an edge have one size), the cube key ->
    // index table and the lattice-vertex key -> slot table with slot -> id
    const uint8_t *mixed = nullptr;
    GsHash hc{nullptr, nullptr, 0};
    GsHash hv{nullptr, nullptr, 0};
    const uint64_t *vslot_id = nullptr;
};
// mixed precision: mark (mark[v] = 1) the corners whose FP32 error could move
// a surface point by more than tol_A or flip a face or fold decision
// adjoint of the triangulation: dL/dp per mesh vertex -> dL/dphi per lattice
// vertex (d_lambda [nlat], overwritten)
int gs_vertex_adjoint(const TriCtx &X, const uint64_t *d_lat_keys, int64_t nlat, const uint64_t *d_mkeys,
                      const double *d_gv, int64_t nm, double *d_lambda, unsigned *d_status, cudaStream_t st);
// volume and area of a closed mesh (d_acc[2]) and their vertex gradients (nullable, accumulated)
int gs_volume_area_dev(const double *d_v, const int32_t *d_tri, int64_t nt, double *d_acc, double *d_gV, double *d_gA,
                       cudaStream_t st);
// adjoint of the field: lambda per lattice vertex -> dL/d(atom centre, radius, D), accumulated
int gs_field_adjoint(const GsProblem &P, const int32_t *d_perm, const uint64_t *d_vkeys, const double *d_lambda,
                     int64_t nv, double *d_gx, double *d_gr, double *d_gD, cudaStream_t st);
__global__ void k_hash_index(GsHash H, const uint64_t *keys, int64_t n, unsigned *status);
// pairs of triangles sharing no vertex that overlap by more than tol (A)
int gs_count_intersections(const double *d_v, int64_t nv, const int32_t *d_t, int64_t nt, double tol,
                           int64_t *n_pairs, cudaStream_t st);
// d_why (nullable) counts the cubes marked through an edge point, a face
// saddle, a fold root, and of those all eight corners; d_in_list (nullable):
// only the n_in listed cubes; d_out_list (nullable, capacity ncubes): the
// cubes that marked a corner, *n_out of them
int gs_tri_marks(const TriCtx &X, const float *d_err, double tol_A, int64_t *d_mark, unsigned long long *d_why,
                 const int64_t *d_in_list, int64_t n_in, int64_t *d_out_list, int64_t *n_out, cudaStream_t st);
// counters: [0] cubes skipped for an inconsistency, [1] degenerate ears, [2] surface cubes
int gs_triangulate(const TriCtx &X, uint64_t **d_tri_keys, int64_t *ntri_total, uint64_t **d_pt_keys,
                   double **d_pt_xyz, int64_t *npt_total, unsigned long long *d_counters, cudaStream_t st);

// launch-shape autotuner (gs_tune.cu): launch(shape, scratch) launches the
// kernel in one of n_choices shapes that compute the same result; scratch
// (non-null during trials: 32 counters whose values are discarded) replaces
// the launch's counters
int gs_tune_run(const char *kernel, int64_t n, int n_choices, cudaStream_t st,
                const std::function<void(int, unsigned long long *)> &launch);

// lattice values within 1e-10 c of c: *d_cnt += their number
int gs_count_near(const double *d_v, int64_t n, double c, unsigned long long *d_cnt, cudaStream_t st);

// copies between device memory and host memory: page-locked mapped host
// buffers through a copy kernel on their device mapping, other host memory
// through cudaMemcpyAsync (gs_scan.cu); gs_host_kind: 0 device, 1 page-locked
// host mapped into the device, 2 other host memory, -1 null
int gs_copy_to_host(void *dst, const void *src, size_t bytes, cudaStream_t st);
int gs_copy_from_host(void *dst, const void *src, size_t bytes, cudaStream_t st);
int gs_host_kind(const void *p);
