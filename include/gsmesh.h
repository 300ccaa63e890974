/*
 * gsmesh.h -- C ABI of the GB300 (sm_103a) Gaussian-surface mesher.
 *
 * The library meshes the level set {x : phi(x) = c} of the Gaussian
 * molecular field phi(x) = sum_i exp(-D (|x - x_i|^2 - r_i^2)) (eq Gaussian1
 * of Liu, Chen & Lu, TMSmesh 2.0) by the paper's two stages: an adaptive
 * partition with per-cube tricubic Legendre estimation (section 2.2) and a
 * per-cube trilinear surface cut into single-valued pieces along fold
 * curves and triangulated by ear clipping (section 2.3).
 *
 * Conventions for every entry point:
 *  - Pointers may be host or device memory (detected per pointer with
 *    cudaPointerGetAttributes); device pointers must be on the current
 *    device.  Inputs are only read; the caller keeps ownership.
 *  - Arrays are C-contiguous: atoms [n][3] FP64 (Angstrom), radii [n] FP64.
 *  - Work is issued on `stream` (a cudaStream_t, NULL = a stream owned by
 *    the library) and the call returns after it has completed.
 *  - Return value 0 on success, a negative GS_ERR_* code otherwise; nothing
 *    is thrown across the ABI.  gs_last_error() gives a message for the
 *    calling thread's last failure.  Output structs are zeroed on error.
 *  - Host waits poll with a deadline (environment GS_WAIT_TIMEOUT_S,
 *    seconds, default 600) and return GS_ERR_TIMEOUT after it; every device
 *    loop is bounded.  A mesh call whose level loop runs out of device
 *    memory or of an internal table is run once more with smaller level
 *    chunks (gs_stats.retries).  For testing these paths, the environment
 *    variable GS_FAULT injects a failure on the host, read at each call:
 *    "alloc@K" (the K-th device allocation fails: GS_ERR_OOM), "capacity@L"
 *    (level L reports a full table on the first attempt: the retry runs),
 *    "timeout" (the first host wait times out: GS_ERR_TIMEOUT).  Nothing is
 *    injected on the device.
 *  - Terms below cutoff_rel * c are dropped: atom i contributes at a point
 *    (a cube) iff the squared distance to the point (to the box) is at most
 *    R_i^2 = r_i^2 - ln(cutoff_rel * c) / D (section 2.2.1, the
 *    neighbourhood truncation after eq polynew).  Default cutoff_rel 1e-8.
 *
 * Key format (64-bit), shared by the mesh output and the parity tests:
 *   bits 0..17 x, 18..35 y, 36..53 z lattice coordinates, 54..58 type,
 *   59..63 level.  Mesh points: type 0..2 = surface point on a cube edge
 *   along axis 0/1/2 (xyz = finest-lattice lower endpoint); 8..19 =
 *   extreme point 8 + 4*axis + 2*side + rank (xyz = finest-lattice lower
 *   corner of the face; side 1 = the fold belongs to the cube on the face's
 *   + side); 20..31 = critical point 20 + 4*(a+b-1) + 2*i + j (xyz =
 *   finest-lattice lower corner of the cube).  Cube keys use type 30 with
 *   the cube's own-level lattice coordinates.
 */
#ifndef GSMESH_H
#define GSMESH_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* status codes */
#define GS_OK 0
#define GS_ERR_ARG (-1)           /* invalid argument (sizes, non-finite values, ranges) */
#define GS_ERR_OOM (-2)           /* device or host allocation failed */
#define GS_ERR_CAPACITY (-3)      /* an internal bound was exceeded (hash full, too many points) */
#define GS_ERR_TIMEOUT (-4)       /* a host wait passed its deadline (GS_WAIT_TIMEOUT_S seconds, default 600) */
#define GS_ERR_CUDA (-5)          /* a CUDA runtime call failed */
#define GS_ERR_DEVICE_STATUS (-6) /* a kernel reported an inconsistency through its status word */

/* precision modes */
#define GS_PREC_FP64 0   /* every field sum and estimate in FP64 (the reference form) */
#define GS_PREC_MIXED 1  /* FP32 compensated sums, FP64 re-evaluation near thresholds; needs D R^2 <= 80
                            for the largest cutoff radius R (R^2 = r^2 - ln(cutoff_rel c)/D), else GS_ERR_ARG */

/* gs_options.child_mode */
#define GS_CHILD_REPROJECT 0
#define GS_CHILD_REEXPAND 1

/* gs_options.decision_order (steps 2 and 3 of section 2.2) */
#define GS_ORDER_BOUNDS_FIRST 0  /* every cube: bound test, then the precision test, then split */
#define GS_ORDER_LITERAL 1       /* a child meeting the precision test is accepted before its bound test; root
                                    cubes that pass the bound test are always divided */

/* gs_options.precision_norm: the size of the higher-than-linear coefficients
   compared with the precision bound (section 2.2.3 leaves the norm open) */
#define GS_NORM_SUM 0  /* sum of their magnitudes (bounds the sup-norm of that part of the polynomial) */
#define GS_NORM_MAX 1  /* largest magnitude */
#define GS_NORM_RSS 2  /* square root of the sum of squares */

/* gs_options.conform_mode: how accepted cubes of different sizes join (section 2.3: the points of the
   neighbouring cubes that lie in the current cube are considered) */
#define GS_CONFORM_CONSTRAIN 0  /* cubes sharing a face or an edge differ by at most one level; a lattice vertex
                                   on a coarser cube's face or edge takes that cube's interpolant, so the
                                   finer and coarser face curves coincide and each takes the other's points;
                                   a vertex whose interpolant and field value lie on different sides of c
                                   splits the coarser cube */
#define GS_CONFORM_EQUAL 1      /* every cube touching a finer one is split until cubes sharing a face or an
                                   edge have one size */

/* gs_options.batch_mode (mesh_gaussian_surface_batch) */
#define GS_BATCH_SHARED_LEVELS 0  /* one level loop per group of molecules with equal D: each kernel of a level
                                     runs once over the octets of all the group's molecules */
#define GS_BATCH_THREADS 1        /* host threads run whole single-molecule meshes on their own streams */

/* decisions reported by gs_cube_decisions */
#define GS_DEC_DISCARD 0
#define GS_DEC_ACCEPT 1
#define GS_DEC_SPLIT 2
#define GS_DEC_FORCED 3  /* accepted at max_depth without meeting the precision bound */

typedef struct {
    int64_t examined[21], discarded[21], accepted[21], forced[21], split[21]; /* per level */
    int64_t pair_terms;        /* (cube, atom) terms inside the cutoff, all levels */
    int64_t vertex_terms;      /* (vertex, atom) terms inside the cutoff */
    int64_t recheck_cubes;     /* cubes re-estimated in FP64 (mixed mode) */
    int64_t recheck_vertices;  /* vertex values re-evaluated in FP64 (mixed mode) */
    int64_t conformity_splits; /* cubes split to equalise levels across faces and edges */
    int64_t n_cubes_final;     /* accepted cubes after conformity */
    int64_t n_cubes_surface;   /* accepted cubes whose corner values straddle c */
    int64_t n_lattice_vertices;
    int64_t n_points;          /* surface points emitted before welding */
    int64_t n_vertices, n_triangles;
    int64_t loop_errors;       /* cubes whose face curves could not be closed */
    int64_t degenerate_ears;   /* ear clipping steps with no strictly valid ear */
    double ms_total, ms_upload, ms_bin, ms_levels, ms_conformity, ms_field, ms_triangulate, ms_weld, ms_download;
    double ms_level[21];
    double ms_accum;           /* summed duration of the tensor-accumulation launches (CUDA events) */
    int64_t n_accum_launches;
    int64_t atom_octets;       /* (octet, atom) pairs whose coefficients were computed */
    int64_t n_kernel_launches; /* this library's kernel launches during the call */
    int64_t recheck_bounds, recheck_precision, recheck_zero; /* mixed mode: why cubes were re-evaluated */
    double mixed_err_ratio;    /* debug bit 0: largest |A_fp32 - A_fp64| / E observed */
    double mixed_band_ratio;   /* debug bit 0: largest |dL|,|dU| / ((dA + 1e-7 sum|A|)(1 + s)) observed */
    int64_t recheck_rank;      /* mixed mode: of recheck_bounds, cubes flagged only through a rank rule near its threshold */
    int64_t vertex_mark_cubes[3]; /* mixed mode: surface cubes whose corners were re-evaluated in FP64 because the
                                     FP32 bound could move an edge point, flip a face saddle, move a fold root */
    int64_t estimate_fast_cubes; /* mixed mode: cubes kept because the corner values of P~ straddle c, decided
                                    without the SVD bounds */
    int64_t constrained_vertices; /* lattice vertices on a coarser cube's face or edge, whose value is that
                                     cube's interpolant (GS_CONFORM_CONSTRAIN) */
    int64_t agreement_splits;     /* cubes split because such an interpolant and the field value lay on
                                     different sides of c */
    int64_t mixed_cubes;          /* final cubes with a neighbour of another size across a face or an edge */
    int64_t retries;              /* 1 when the level loop ran out of device memory or of an internal table and
                                     the call was run again with smaller level chunks */
    int64_t near_threshold[4];    /* decisions taken in FP64 whose margin was below 1e-10 relative: [0] bound
                                     test, min(c-L, U-c) against |c|+|L|+|U|; [1] precision test, |precision -
                                     sum|high|| against their sum; [2] a 99% rank rule, |sum_{i<=j} s_i - 0.99
                                     sum s| against sum s; [3] lattice vertices with |value - c| < 1e-10 c.  Such
                                     a decision may differ from an independent FP64 evaluation by rounding
                                     alone (the oracle resolves them in quad precision) */
    int64_t refine_vertices;      /* mixed mode: lattice vertex values re-evaluated in double-word FP32 (a hi + lo
                                     float pair per value; bound about 1e-10 relative) where the FP32 bound was
                                     too wide; recheck_vertices counts those that then went on to FP64 */
    int64_t vertex_mark_all;      /* mixed mode: of vertex_mark_cubes, cubes with all eight corners marked */
    int64_t vertex_mark_fp64_cubes[3]; /* mixed mode: cubes marked again with the double-word bounds (edge point,
                                     face saddle, fold root), whose corners were re-evaluated in FP64 */
} gs_stats;

typedef struct {
    double min_edge;        /* finest cube edge (A); default 0.25 */
    int precision_mode;     /* GS_PREC_FP64 (default) or GS_PREC_MIXED */
    double cutoff_rel;      /* default 1e-8 */
    void *cuda_stream;      /* cudaStream_t or NULL */
    int device_output;      /* 1: out arrays stay on the device (free with mesh_free) */
    int debug_flags;        /* bit 0: mixed mode also runs FP64 on every cube and counts disagreements;
                               bit 1: process each level in chunks of 1000 parent octets (instead of 2^21),
                               so that small inputs take the multi-chunk path of large ones */
    gs_stats *stats;        /* nullable: filled on success */
    int child_mode;         /* child tensors: GS_CHILD_REPROJECT (default: projected from the atoms on each
                               child box) or GS_CHILD_REEXPAND (the parent's polynomial re-expanded on the
                               child; the other reading of eq childtensor; FP64 form only) */
    int decision_order;     /* GS_ORDER_BOUNDS_FIRST (default) or GS_ORDER_LITERAL (FP64 form only) */
    int precision_norm;     /* GS_NORM_SUM (default), GS_NORM_MAX or GS_NORM_RSS (FP64 form only) */
    int conform_mode;       /* cubes of different sizes: GS_CONFORM_CONSTRAIN (default) or GS_CONFORM_EQUAL */
    int batch_mode;         /* mesh_gaussian_surface_batch: GS_BATCH_SHARED_LEVELS (default) or GS_BATCH_THREADS */
} gs_options;

typedef struct {
    double *vertices;       /* [n_vertices][3] FP64, A */
    int64_t n_vertices;
    int32_t *triangles;     /* [n_triangles][3], counter-clockwise seen from outside (phi < c) */
    int64_t n_triangles;
    uint64_t *vertex_keys;  /* [n_vertices] canonical keys (see above) */
    uint64_t *cube_keys;    /* [n_cubes] accepted cubes after conformity */
    int64_t n_cubes;
    int on_device;          /* arrays are device memory */
    int64_t mismatches;     /* debug bit 0: mixed-vs-FP64 decision disagreements outside the band */
} gs_mesh;

/* gs_options with the defaults above */
gs_options gs_default_options(void);

/*
 * mesh_gaussian_surface -- mesh {phi = c} (eqs Gaussian1, polynew, bound2,
 * bound3, linear1, intersection, curve, fold1, critical; sections 2.2-2.3).
 *   atoms     [n_atoms][3] centres, radii [n_atoms] (host or device)
 *   D > 0 decay rate, c > 0 isovalue, precision > 0 bound on the sum of the
 *   absolute higher-than-linear Legendre coefficients (section 2.2.3),
 *   max_depth in [0, 20]: the root grid has edge min_edge * 2^max_depth and
 *   cubes are refined at most max_depth times.
 *   opt may be NULL (defaults).  On success *out holds library-allocated
 *   arrays; release them with mesh_free.  An empty surface (every cube
 *   discarded) is a success with zero triangles.
 * Errors: GS_ERR_ARG for n_atoms <= 0, non-finite or negative inputs, D, c or
 * precision <= 0, max_depth outside [0,20], or a lattice wider than 2^18
 * points per axis; GS_ERR_OOM, GS_ERR_CAPACITY, GS_ERR_CUDA,
 * GS_ERR_DEVICE_STATUS as above.
 */
int mesh_gaussian_surface(const double *atoms, const double *radii, int64_t n_atoms, double D, double c,
                          double precision, int max_depth, const gs_options *opt, gs_mesh *out);

/* Output buffers owned by the caller (host memory, pinned or pageable, or
 * device memory, told apart by the CUDA runtime): the mesh is copied into
 * them directly, so buffers kept across calls (pinned host memory for a
 * host consumer) avoid a per-call allocation and staging copy. */
typedef struct {
    double *vertices;       /* [cap_vertices][3] */
    int32_t *triangles;     /* [cap_triangles][3] */
    uint64_t *vertex_keys;  /* [cap_vertices] or NULL (not wanted) */
    uint64_t *cube_keys;    /* [cap_cubes] or NULL (not wanted) */
    int64_t cap_vertices, cap_triangles, cap_cubes;
    int64_t n_vertices, n_triangles, n_cubes;   /* out: the mesh's sizes (also on GS_ERR_CAPACITY) */
} gs_mesh_buffers;

/*
 * mesh_gaussian_surface_into -- mesh_gaussian_surface with the result copied
 * into caller-owned buffers (layout and order as in gs_mesh).  On success the
 * n_* fields hold the sizes.  When a buffer is smaller than the mesh the call
 * writes nothing into the buffers, sets the n_* fields to the sizes needed
 * and returns GS_ERR_CAPACITY; the caller may grow the buffers and call
 * again.  Other errors as mesh_gaussian_surface; GS_ERR_ARG also for a
 * negative capacity or a NULL vertices/triangles buffer with a positive
 * capacity.
 */
int mesh_gaussian_surface_into(const double *atoms, const double *radii, int64_t n_atoms, double D, double c,
                               double precision, int max_depth, const gs_options *opt, gs_mesh_buffers *out);

/*
 * mesh_gaussian_surface_batch -- mesh n_mols independent molecules (the
 * method applies to each molecule on its own; the paper meshes one at a
 * time).  Molecule m is atoms[offsets[m] .. offsets[m+1]) with decay rate
 * D[m]; c, precision, max_depth and opt are shared (opt->stats and
 * opt->cuda_stream are ignored).  out [n_mols] receives one mesh per
 * molecule, each identical to what mesh_gaussian_surface gives for that
 * molecule alone (release each with mesh_free); stats [n_mols] (nullable)
 * one record per molecule.
 *   offsets [n_mols + 1] host int64, offsets[0] = 0, strictly increasing;
 *   D [n_mols] host.  Atoms and radii host or device.
 * opt->batch_mode:
 *   GS_BATCH_SHARED_LEVELS (default; GS_CHILD_REPROJECT only, else as
 *   GS_BATCH_THREADS): the molecules are grouped by D.  Per group one level
 *   loop (section 2.2) runs each kernel of a level once over the octets of
 *   all its molecules; every octet carries its molecule's index, and a
 *   device table holds each molecule's atoms, cell list and root grid.  The
 *   host reads one block of per-molecule counts per level and group.  Then
 *   n_workers host threads, each with its own stream, finish the meshes
 *   (conformity, lattice, field, triangulation, weld), largest first.  In
 *   stats, examined .. split are the molecule's own; pair_terms,
 *   atom_octets, recheck_cubes, the recheck reasons, estimate_fast_cubes,
 *   ms_level, ms_levels and ms_accum are those of its group; ms_total
 *   covers the molecule's own stages after the level loop.
 *   GS_BATCH_THREADS: n_workers host threads run whole single-molecule
 *   meshes on their own streams, largest molecules first.
 * Errors: as mesh_gaussian_surface for any molecule (the message names it);
 * GS_ERR_ARG for an unknown batch_mode; on error every out[m] is released
 * and zeroed.
 */
int mesh_gaussian_surface_batch(const double *atoms, const double *radii, const int64_t *offsets, int64_t n_mols,
                                const double *D, double c, double precision, int max_depth, const gs_options *opt,
                                int n_workers, gs_mesh *out, gs_stats *stats);

/* release the arrays of a gs_mesh (host or device) and zero it; NULL-safe */
void mesh_free(gs_mesh *m);

/* static description of a status code */
const char *gs_status_string(int status);

/* message for the calling thread's last failure ("" if none) */
const char *gs_last_error(void);

/*
 * Launch-shape autotuner.  Kernels with several launch shapes that compute
 * the same result (the lattice-field kernel's tile: warps per block and
 * vertices per lane; the FP32 tensor accumulation's grid size) time every
 * shape on the first call's own data for each size class (a power of two of
 * the item count), keep the fastest for the process, and launch it from
 * then on.  Results do not depend on the choice.  GS_AUTOTUNE=0
 * (environment) turns tuning off (shape 0 everywhere); GS_AUTOTUNE=shape:K
 * takes shape K everywhere (the last shape where a kernel has fewer).
 * gs_autotune_report writes one line per (kernel, size class): "kernel 2^k
 * choice t0 t1 ..." (trial milliseconds per shape) into buf [cap] (NUL-
 * terminated, cut to fit; buf may be NULL) and returns the length the
 * whole report needs, NUL included.  gs_autotune_reset forgets every
 * choice.  Both are thread-safe.
 */
int64_t gs_autotune_report(char *buf, int64_t cap);
void gs_autotune_reset(void);

/* how the library sees a buffer: 0 device memory, 1 page-locked host memory
 * mapped into the device (the library moves meshes into it with a copy
 * kernel at the rate of the host link), 2 other host memory (pageable:
 * cudaMemcpyAsync, staged by the runtime), -1 NULL.  A query only; no
 * device work. */
int gs_memory_kind(const void *p);

/* sizeof of the ABI structs (0: gs_stats, 1: gs_options, 2: gs_mesh; else -1),
 * for bindings to verify their layouts */
int64_t gs_struct_size(int which);

/*
 * gs_bin_atoms -- uniform cell list by a stable counting sort (the
 * neighbourhood search behind the truncation of section 2.2.1).
 *   cell = floor((x - origin) / cell_size) per axis, clamped to [0, dims-1],
 *   linear index x + dims[0] * (y + dims[1] * z).
 *   cell_start [dims0*dims1*dims2 + 1] int32: atoms of cell k are
 *   atom_perm[cell_start[k] .. cell_start[k+1]), in ascending atom index.
 *   All arrays host or device; outputs are written where they live.  The
 *   time is bounded by n_atoms however the atoms crowd into cells.
 */
int gs_bin_atoms(const double *atoms, int64_t n_atoms, double cell_size, const double *origin,
                 const int64_t *dims, int32_t *cell_start, int32_t *atom_perm, void *stream);

/*
 * gs_bin_atoms_static -- the same cell list as gs_bin_atoms, for callers that
 * cannot let the library allocate memory: programs that give all device
 * memory to their own allocator at start-up (a framework's caching pool, a
 * fixed-budget service) or cannot afford the device-wide synchronisation a
 * cudaMalloc or cudaFree may cause mid-run.  The paper has no counterpart;
 * this is a deployment variant of the binning step.
 *   atoms [n_atoms][3], cell_start [dims0*dims1*dims2 + 1] and atom_perm
 *   [n_atoms] must be device memory on the current device; origin [3] and
 *   dims [3] are host arrays.  Same results as gs_bin_atoms.
 *   Limits: n_atoms <= GS_STATIC_MAX_ATOMS, cells <= GS_STATIC_MAX_CELLS;
 *   larger requests, host pointers, memory of another device or NULLs
 *   return GS_ERR_ARG.  Buffer lengths cannot be checked through plain
 *   pointers: shorter buffers than the above are the caller's error (the
 *   Python binding checks them).  The time is bounded by n_atoms however
 *   the atoms crowd into cells (stable radix passes, no per-cell sort).
 *   No cudaMalloc, cudaFree or allocating library call is made: the
 *   temporaries live in one fixed device array (about 18 MB, reserved on
 *   every GPU that loads the library until the process exits).  Every call
 *   shares that array; calls whose work overlaps on the GPU race and give
 *   wrong results.  The first call on a device looks up the array's address
 *   (once per device).  Work runs on `stream` (NULL: the legacy default
 *   stream) and the call returns after it has completed: it waits on the
 *   stream, so it cannot be captured into a CUDA graph.
 */
#define GS_STATIC_MAX_ATOMS (1 << 20)
#define GS_STATIC_MAX_CELLS (1 << 20)
int gs_bin_atoms_static(const double *atoms, int64_t n_atoms, double cell_size, const double *origin,
                        const int64_t *dims, int32_t *cell_start, int32_t *atom_perm, void *stream);

/*
 * gs_eval_field -- phi and grad phi at points (eq Gaussian1 with the
 * truncation above).  points [n_points][3], phi [n_points], grad
 * [n_points][3] (nullable).  precision_mode as in gs_options.
 */
int gs_eval_field(const double *atoms, const double *radii, int64_t n_atoms, double D, double c,
                  double cutoff_rel, const double *points, int64_t n_points, double *phi, double *grad,
                  int precision_mode, void *stream);

/*
 * gs_eval_field_bounded -- phi at points in double-word FP32 (each value a hi
 * + lo float pair: the evaluation the mixed mode uses where an FP32 bound is
 * too wide), with an upper bound err[i] of |phi[i] - phi_exact| (eq Gaussian1
 * with the truncation above; the terms are those of the FP64 form).
 * points [n_points][3], phi [n_points] FP64, err [n_points] FP32; host or
 * device pointers (all of one kind per array), not retained.  Needs D R^2 <=
 * 80 (R the largest cutoff radius), else GS_ERR_ARG.
 */
int gs_eval_field_bounded(const double *atoms, const double *radii, int64_t n_atoms, double D, double c,
                          double cutoff_rel, const double *points, int64_t n_points, double *phi, float *err,
                          void *stream);

/*
 * gs_cube_decisions -- coefficient tensor A (eqs polynew, tensor1, tensor2),
 * bounds (eqs SVD1-SVD7, bound1-bound3) and decision for listed cubes of the
 * problem's root lattice (keys of type 30 at their level).  A [n][64] in
 * (j,k,l) order with j <-> x (nullable), bounds [n][6] = (L, U, sum|R|,
 * sum|high|, rank, sum of inner ranks) (nullable), dec [n] int32.
 */
int gs_cube_decisions(const double *atoms, const double *radii, int64_t n_atoms, double D, double c,
                      double precision, double min_edge, int max_depth, double cutoff_rel,
                      const uint64_t *cube_keys, int64_t n_cubes, double *A, double *bounds, int32_t *dec,
                      int precision_mode, void *stream);

/*
 * gs_triangulate_grid -- the section 2.3 triangulation of a uniform grid of
 * given corner values (every cube accepted at one level, unit spacing,
 * origin 0): values [(nz+1)][(ny+1)][(nx+1)], x fastest.  Output as for
 * mesh_gaussian_surface (opt: stream and device_output are honoured).
 */
int gs_triangulate_grid(int64_t nx, int64_t ny, int64_t nz, const double *values, double c,
                        const gs_options *opt, gs_mesh *out);

/*
 * gs_mesh_backward -- adjoint of mesh_gaussian_surface: given dL/dp for every
 * vertex of the mesh that mesh_gaussian_surface returns for the same
 * arguments, accumulate dL/d(atom centres), dL/d(radii) and dL/dD.  The cube
 * set and the topology are held fixed (the derivative of the piecewise
 * smooth map); every vertex is differentiated through the corner values it
 * is computed from -- edge points through eq intersection, extreme points
 * through the fold equations eq fold1 by implicit differentiation, critical
 * points (eq critical) through the two fold roots that define them -- and
 * the corner values through eq Gaussian1 (terms recomputed, not stored).
 * The paper defines no derivatives; this is the chain rule applied to its
 * construction.  The mesh is recomputed inside the call.
 *   grad_vertices [n_vertices][3] (host or device), in the mesh's vertex order;
 *   n_vertices must equal the mesh's vertex count (else GS_ERR_ARG).
 *   grad_atoms [n_atoms][3], grad_radii [n_atoms], grad_D [1] (host or device,
 *   each nullable), overwritten.  FP64 atomics: sums are reproducible only up
 *   to rounding order.  Errors as mesh_gaussian_surface; GS_ERR_DEVICE_STATUS
 *   if a vertex key does not resolve to its cube or edge.
 */
int gs_mesh_backward(const double *atoms, const double *radii, int64_t n_atoms, double D, double c,
                     double precision, int max_depth, const gs_options *opt, const double *grad_vertices,
                     int64_t n_vertices, double *grad_atoms, double *grad_radii, double *grad_D);

/*
 * gs_volume_area -- enclosed volume sum p0.(p1 x p2)/6 and surface area
 * sum |(p1 - p0) x (p2 - p0)|/2 of a closed mesh with outward (counter-
 * clockwise seen from outside) triangles, the two measures the paper
 * reports for its meshes (section 3.4), with their gradients per vertex.
 *   vertices [n_vertices][3], triangles [n_triangles][3] int32 (host or
 *   device); volume_area [2] out; grad_volume, grad_area [n_vertices][3]
 *   (nullable) overwritten.  GS_ERR_ARG if a triangle index is outside
 *   [0, n_vertices).  opt: only the stream is used (NULL: a private stream).
 */
int gs_volume_area(const double *vertices, int64_t n_vertices, const int32_t *triangles, int64_t n_triangles,
                   double *volume_area, double *grad_volume, double *grad_area, const gs_options *opt);

/*
 * gs_mesh_intersections -- number of pairs of triangles that share no vertex
 * and overlap by more than tol (A) along every separating axis of the pair
 * (the paper's count of intersecting triangle pairs, section 3.2, which it
 * reports as zero for its meshes).  vertices [n_vertices][3], triangles
 * [n_triangles][3] int32, host or device.  GS_ERR_ARG if a triangle index
 * is outside [0, n_vertices) or tol < 0.
 */
int gs_mesh_intersections(const double *vertices, int64_t n_vertices, const int32_t *triangles,
                          int64_t n_triangles, double tol, int64_t *n_pairs, const gs_options *opt);

#ifdef __cplusplus
}
#endif

#endif /* GSMESH_H */
