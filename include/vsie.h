/*
 * vsie.h -- C ABI of libvsie: the matrix-free apply and GMRES solve of the discretised
 * nested volume-surface integral equation (VSIE) for heterogeneous acoustic
 * transmission problems, on one NVIDIA B300 (sm_103a).
 *
 * Operator (Eq. vsie, Theorem "VSIE", with the block system of Sec. 2.3 "Linear
 * system"): for every collocation point x_i (tetrahedron centroids, then interface
 * triangle centroids)
 *
 *   (A p)_i = m_i p_i
 *           - sum_e int_e G(x_i,y) (beta - k0^2 alpha)_e dy p_e          (single layer V)
 *           + sum_e div_x int_e G(x_i,y) grad(alpha)_e dy p_e            (adjoint DL, T)
 *           + sum_t int_t dG(x_i,y)/dn_y omega_t dS_y p_t                (double layer K)
 *
 * G = exp(i k0 r)/(4 pi r) (Eq. greens_function), alpha = rho0/rho - 1 (Eq. alpha),
 * beta = (rho0/rho)(omega/c)^2 - (omega/c0)^2 (Eq. beta), m from Eq. (mass_function),
 * omega_t = alpha_1 on Gamma_1 and alpha_2 - alpha_1 on Gamma_2.  P0 unknowns with point
 * collocation (Sec. 2.3.4).  Time convention e^{-i omega t}.
 *
 * Conventions shared by every call:
 *  - Unknown order: [tetrahedra in input order | triangles in input order]; n = n_tet + n_tri.
 *  - Complex vectors are interleaved (re, im) float64, i.e. C99 double _Complex /
 *    torch.complex128.  Multi-RHS blocks are column-major n x nrhs (column j at x + 2*n*j).
 *  - Pointers named d_* are DEVICE pointers on the handle's device, caller-owned; the
 *    library never frees them.  Pointers named h_* are host pointers, caller-owned.
 *  - ``stream`` is a cudaStream_t passed as void* (NULL = legacy default stream).  Calls
 *    are asynchronous with respect to the host unless stated otherwise; all work of a
 *    handle must be issued on one stream at a time.
 *  - No exception crosses the ABI: every call returns a vsie_status; on error
 *    vsie_last_error() holds a message (thread-local) and outputs are unspecified.
 */
#ifndef VSIE_H
#define VSIE_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  VSIE_OK = 0,
  VSIE_ERR_ARG = 1,           /* invalid argument (null pointer, size, option)          */
  VSIE_ERR_MESH = 2,          /* degenerate element, index out of range                 */
  VSIE_ERR_CUDA = 3,          /* a CUDA runtime call failed                             */
  VSIE_ERR_OOM = 4,           /* device allocation failed                               */
  VSIE_ERR_NOT_CONVERGED = 5, /* solver stopped at its iteration limit (x still written) */
  VSIE_ERR_BREAKDOWN = 6,     /* Krylov breakdown with a nonzero residual               */
  VSIE_ERR_NAN = 7            /* non-finite input or intermediate value                 */
} vsie_status;

typedef struct vsie_handle vsie_handle; /* opaque, library-owned */

/* Geometry of Omega_1, Omega_2, Gamma_1, Gamma_2 (Sec. 2.1, Fig. 1).  Host arrays,
 * caller-owned, copied during vsie_create. */
typedef struct {
  int64_t n_vert;
  const double* vert;       /* 3*n_vert, xyz per vertex                               */
  int64_t n_tet;
  const int32_t* tet;       /* 4*n_tet vertex indices (any orientation)               */
  int64_t n_tri;
  const int32_t* tri;       /* 3*n_tri vertex indices; (b-a)x(c-a) must point out of
                               the subdomain the interface encloses (n_1 on Gamma_1,
                               n_2 on Gamma_2)                                        */
} vsie_mesh;

/* Material (Eqs. density, speed_of_sound): per-tetrahedron values and the one-sided
 * density limits on every interface triangle.  Host arrays, caller-owned, copied. */
typedef struct {
  double rho0, c0;          /* exterior density and speed of sound                    */
  const double* rho;        /* n_tet, > 0                                             */
  const double* c;          /* n_tet, > 0                                             */
  const double* grad_alpha; /* 3*n_tet gradient of alpha per tetrahedron, or NULL for
                               a piecewise-constant density (adjoint DL term absent)  */
  const double* tri_rho_in; /* n_tri: density limit on the side the normal leaves    */
  const double* tri_rho_out;/* n_tri: density limit on the side the normal enters
                               (rho0 on Gamma_1, rho_1 on Gamma_2)                    */
} vsie_material;

/* Discretisation options (readings of Sec. 2.3.4 for tetrahedra and flat triangles). */
typedef struct {
  int32_t tet_far_points;   /* 1: centroid rule in the far field; 4: the degree-2
                               four-point rule on every tetrahedron                   */
  double near_radius;       /* with tet_far_points == 1: tetrahedra whose centroid is
                               closer than this to a target use the four-point rule   */
  double tri_near_radius;   /* triangles whose centroid is closer than this to a target
                               use the singularity-subtracted rule (exact Laplace
                               solid angle + three-point Helmholtz remainder); 0 = off */
  int32_t tile_override;    /* 0 = library default launch shape                       */
  int32_t debug_flags;      /* 0 in normal use.  Bit 0 (failure-path testing): the
                               tensor-core kernel of vsie_apply_batched never starts its
                               bulk copies, so its bounded waits expire and the call
                               returns VSIE_ERR_CUDA without faulting the device      */
} vsie_options;

/* Build the discrete operator on the current CUDA device: element geometry, material
 * weights, far-field source points and the FP64 near-field/self correction matrix
 * (computed on the device).  k0 = omega/c0 > 0 is the exterior wavenumber.  Blocking.
 * Errors: VSIE_ERR_ARG (null/size), VSIE_ERR_MESH (index out of range, zero-volume
 * element, non-positive material), VSIE_ERR_OOM, VSIE_ERR_CUDA. */
vsie_status vsie_create(const vsie_mesh* mesh, const vsie_material* mat, double k0,
                        const vsie_options* opt, vsie_handle** out);

/* Nonuniform cuboid grid (Sec. 2.3.4, "Computational domain"): nx x ny x nz cells
 * [x_i, x_{i+1}] x [y_j, y_{j+1}] x [z_k, z_{k+1}]; every cell face meets exactly one
 * neighbouring face (no hanging nodes), so interfaces that follow cell faces are matched. */
typedef struct {
  int32_t nx, ny, nz;
  const double* x_edges;    /* nx + 1 strictly increasing coordinates */
  const double* y_edges;    /* ny + 1 */
  const double* z_edges;    /* nz + 1 */
} vsie_cuboid_grid;

/* Build the operator of the paper's own discretisation (Sec. 2.3.4, "Discrete
 * representation"): P0 unknowns on the cells and on the rectangular faces across which
 * the density jumps, collocation at the centroids, every integral by the midpoint rule, the
 * single-layer self term over the ball of equal volume (the double-layer self term of a
 * flat face is 0).  rho, c: host nx*ny*nz per-cell density and sound speed, cell (i, j, k)
 * at (i ny + j) nz + k; rho0, c0: the exterior material (also the material outside the
 * grid); k0 = omega/c0.  Unknown order: the cells, then the jump faces normal to x (face a
 * between cells a-1 and a, a = 0..nx, outside the grid the exterior density), ordered by
 * (a, j, k), then those normal to y by (i, b, k), then those normal to z by (i, j, c);
 * a face's normal is the +axis direction, its "in" side the cell below.  The handle
 * serves every entry point of the tetrahedral one; the field-point near rules are off.
 * Blocking.  Errors: VSIE_ERR_ARG (null/size), VSIE_ERR_MESH (edges not increasing,
 * non-positive material), VSIE_ERR_OOM, VSIE_ERR_CUDA. */
vsie_status vsie_create_cuboid(const vsie_cuboid_grid* grid, const double* rho, const double* c,
                               double rho0, double c0, double k0, vsie_handle** out);

/* The interface unknowns of a cuboid grid, host-only (no device work): the faces across
 * which the density jumps, in the unknown order of vsie_create_cuboid (they follow the
 * nx*ny*nz cells).  n_faces receives their number; the arrays, each NULL or of at least
 * `capacity` entries (centres 3 per face), receive per face its centre, normal axis
 * (0, 1, 2: the normal is that +axis), area, omega = alpha_in - alpha_out = rho0/rho_in -
 * rho0/rho_out (Eq. vsie) and mass function (rho0/rho_in + rho0/rho_out)/2 (Eq.
 * mass_function).  Call with capacity 0 and NULL arrays to count.  VSIE_ERR_ARG on a
 * null argument or a capacity below the count with arrays given; VSIE_ERR_MESH on edges
 * that do not increase or a non-positive density. */
vsie_status vsie_cuboid_faces(const vsie_cuboid_grid* grid, const double* rho, double rho0,
                              int64_t capacity, int64_t* n_faces, double* centres, int32_t* axis,
                              double* area, double* omega, double* mass);

/* Change the frequency of an existing operator: k0 = omega/c0 enters the volume weights
 * through beta (Eq. beta) and every pair through G = exp(i k0 r)/(4 pi r) (Eq.
 * greens_function), so the weights, source records and the near/self correction are
 * rebuilt from the creation inputs (kept on the host by vsie_create / vsie_create_cuboid)
 * exactly as a new create at k0 would build them; the geometry, material and the work
 * shapes chosen by vsie_autotune stay.  Blocking (synchronises the device first).
 * Every device buffer of the handle is reallocated, so CUDA-graph plans recorded on it
 * (vsie_graph_create_batched) must be recreated.  On an error other than VSIE_ERR_ARG the
 * handle is left empty (n = 0, no device buffers): it may be destroyed, or rebuilt by
 * another vsie_set_frequency. */
vsie_status vsie_set_frequency(vsie_handle* h, double k0);

void vsie_destroy(vsie_handle* h);

/* Sizes of the discrete system: n unknowns (volume elements, then interface elements),
 * the number of far-field source points (quadrature points of the far rule), and the
 * entries of the near/self correction.  Any output may be NULL.  VSIE_ERR_ARG on a null
 * handle. */
vsie_status vsie_sizes(const vsie_handle* h, int64_t* n, int64_t* n_far_sources,
                       int64_t* nnz_correction);

/* y = A x for nrhs columns (Eq. vsie at every collocation point).  precision 32: far-field
 * sums in FP32 with per-tile FP64 accumulation, correction and mass in double-float/FP64;
 * precision 48: far-field sums in double-float arithmetic on the FP32 pipe (about 2^-47
 * per operation, FP64-class results); precision 64: everything in FP64.  x, y: device
 * complex128, n x nrhs column-major, must not alias.  Asynchronous.  Errors: VSIE_ERR_ARG
 * (null pointer, nrhs < 1, precision not 32/48/64, aliasing), VSIE_ERR_OOM,
 * VSIE_ERR_CUDA. */
vsie_status vsie_apply(vsie_handle* h, const void* d_x, void* d_y, int32_t nrhs,
                       int32_t precision, void* stream);

/* Same operator with host buffers: copies x to the device, applies, copies y back and
 * synchronises the stream before returning.  h_x, h_y: host complex128 n x nrhs
 * (interleaved doubles), caller-owned; pinned memory makes the copies asynchronous with
 * respect to other streams.  Uses library-owned device buffers, grown on demand.  Errors
 * as vsie_apply. */
vsie_status vsie_apply_host(vsie_handle* h, const double* h_x, double* h_y, int32_t nrhs,
                            int32_t precision, void* stream);

/* Rows row_begin .. row_end-1 of y = A x (Eq. vsie at those collocation points only):
 * d_y[i - row_begin] = (A x)_i.  Every far-field source point contributes to every row,
 * so x holds all n unknowns while y holds only the rows.  Rows are independent and equal in
 * far-field work; a contiguous split of 0..n over several devices therefore
 * partitions an apply, each device holding the whole operator and all of x (the row-sharded
 * multi-GPU apply gathers the slices).  Each row equals the same row of vsie_apply to
 * rounding; the summation order differs.  The same call also gives the error or the rate
 * of an apply on a sample of rows.  x: device complex128 n; y: device complex128
 * (row_end - row_begin); they must not alias.  precision 32, 48 or 64 as in vsie_apply.
 * Asynchronous; may grow the handle's scratch on first use.  Errors: VSIE_ERR_ARG (null
 * pointer, aliasing, precision, rows outside 0 <= row_begin <= row_end <= n),
 * VSIE_ERR_OOM, VSIE_ERR_CUDA. */
vsie_status vsie_apply_rows(vsie_handle* h, const void* d_x, void* d_y, int64_t row_begin,
                            int64_t row_end, int32_t precision, void* stream);

/* One vsie_apply (nrhs = 1) with CUDA events recorded on ``stream`` between its phases;
 * blocks until done.  kernel_ms[4] receives the device time of: the charge prescale, the
 * far-field sum over volume sources without a vector weight, the far-field sum over
 * sources with a vector weight (interfaces, heterogeneous density), and the correction
 * + mass kernel.  The phases run one after the other here even where vsie_apply runs the
 * G and K sums concurrently (vsie_set_tuning, vsie_autotune).  *launches (optional)
 * receives the number of kernels one vsie_apply launches with the work shapes in use. */
vsie_status vsie_apply_timed(vsie_handle* h, const void* d_x, void* d_y, int32_t precision,
                             void* stream, double* kernel_ms, int32_t* launches);

/* y = A x like vsie_apply, for callers that may not allocate device memory once set-up
 * is over: a host application that hands all device memory to its own pool at start-up
 * and accounts for every later byte, or a latency-critical loop that must not pay the
 * implicit device synchronisation of cudaMalloc.  (The paper has no counterpart; this is
 * an interface concern of the library.)  vsie_apply may grow a device buffer on first use
 * for source-split partial sums; this variant keeps them in a fixed device array of
 * 2,097,152 complex128 elements (32 MiB) compiled into the library, which every GPU that
 * loads the library holds until the process exits.  Calls allocate nothing and free
 * nothing.  The array's device address is looked up (and the array loaded on the device,
 * with the library's device code) once per device, when an operator is created there;
 * should that lookup fail, the first call on the device repeats it (with the handle's
 * device made current) and reports the failure, so make that first call before any
 * stream capture.  A device reset (cudaDeviceReset) reloads the library's device code
 * and leaves the kept address stale: do not use this call on a device after resetting
 * it.  All calls share the one array and its contents persist between calls (every
 * element a call reads it has written first), so calls that overlap on the GPU -- on
 * different streams or different handles -- race and must be serialised by the caller.
 * Same arguments, layouts and precisions as vsie_apply.  Errors: VSIE_ERR_ARG when the
 * operator's launch shape at the requested precision needs more scratch than the array
 * holds (the message gives both sizes; y is not written; vsie_apply still works), and as
 * vsie_apply otherwise. */
vsie_status vsie_apply_noalloc(vsie_handle* h, const void* d_x, void* d_y, int32_t nrhs,
                               int32_t precision, void* stream);

/* y = A x for a block of nrhs right-hand sides (Eq. vsie at every collocation point, as
 * vsie_apply) with the far-field sums over volume and interface sources computed once per
 * kernel value for 64 columns at a time.
 *   precision 32: each tile of kernel values is evaluated in FP32 and contracted with the
 *     charge columns on the tensor cores (three-term TF32 split, FP32 accumulation of one
 *     32-source tile at a time, compensated running sum, FP64 output);
 *   precision 64: every kernel value is evaluated in FP64 on the CUDA cores and applied
 *     to the 64 columns in FP64 (the residual operator of vsie_solve_batched).
 * Volume sources with grad(alpha) != 0, the correction and the mass use the per-column
 * path of the same precision.  Same layouts as vsie_apply.  Blocks until done (precision
 * 32 reads the tensor-core kernels' timeout flag).  Errors: VSIE_ERR_ARG, VSIE_ERR_OOM,
 * VSIE_ERR_CUDA (also when a bounded wait in the tensor-core kernel expired). */
vsie_status vsie_apply_batched(vsie_handle* h, const void* d_x, void* d_y, int32_t nrhs,
                               int32_t precision, void* stream);

/* Autotuning of the work shapes (the target-tile x source-chunk items of the persistent
 * kernels) on this operator.  flags bit 0: the FP32 far-field sums of vsie_apply (sources
 * per work item in {512, 1024, 2048, 4096} x resident blocks per SM in {max, 3/4 max,
 * max/2}, per source class; then whether the volume (G) and interface (K) sums run one
 * after the other or concurrently on two streams, each with part of every SM's resident
 * blocks, so that the MUFU-bound G sum and the FMA-bound K sum share the SMs' pipes);
 * bit 1: the tensor-core sums of vsie_apply_batched (32-source
 * tiles per work item in {16, 32, 64, 128}).  Each candidate is timed (CUDA events, best
 * of two runs after a warm-up) on a sample of the targets sized to a few tens of
 * milliseconds, with pseudo-random charges; the fastest is kept in the handle and used
 * by every later call (results change only by the summation order).  Allocates and frees
 * temporary buffers (2 x n x 64 complex128 with bit 1); blocking.  report: NULL or the
 * chosen shapes with their times and the built-in defaults' times on the same sample. */
typedef struct {
  int32_t far_chunk[3];          /* G, K, F classes: sources per work item (0: class absent) */
  int32_t far_blocks_per_sm[3];  /* resident blocks per SM */
  double far_ms[3];              /* chosen shape, ms on the tuning sample */
  double far_default_ms[3];      /* built-in default shape (1024, max), same sample */
  int32_t batch_chunk_tiles;     /* tensor-core sums: 32-source tiles per work item */
  double batch_ms;               /* chosen, ms for G + K on the tuning sample (64 columns) */
  double batch_default_ms;       /* built-in default (64 tiles) */
  int32_t candidates;            /* configurations timed */
  int32_t gk_blocks_per_sm[2];   /* G and K sums run concurrently with these blocks per SM
                                    each; 0, 0: one after the other (bit 0) */
  double gk_ms;                  /* chosen, ms for G + K on the tuning sample */
  double gk_sequential_ms;       /* G then K with their tuned shapes, same sample */
} vsie_tuning;
vsie_status vsie_autotune(vsie_handle* h, int32_t flags, vsie_tuning* report, void* stream);

/* The work shapes in use (times zero): the fields vsie_set_tuning reads, 0 where the
 * built-in default applies.  Errors: VSIE_ERR_ARG for a null argument. */
vsie_status vsie_get_tuning(const vsie_handle* h, vsie_tuning* tuning);

/* Sets the work shapes without timing them, e.g. those an earlier vsie_autotune chose for the
 * same mesh (read back with vsie_get_tuning): far_chunk (0 or a multiple of 128, at most
 * 2^20) and far_blocks_per_sm (0..64, clamped to the kernel's occupancy) per class,
 * batch_chunk_tiles (0..65536) and gk_blocks_per_sm (both 0: the G and K sums one after
 * the other; both >= 1: concurrently with that many blocks per SM each); 0 selects the
 * built-in default; the time fields are ignored.  Allocates the concurrent sums' buffers (a
 * second stream, two events, n complex128 values and split slots) the first time they are
 * chosen; blocking only for those allocations.  Results change only by the summation order.
 * Errors: VSIE_ERR_ARG for a null argument or a value out of range (the handle unchanged);
 * VSIE_ERR_CUDA if an allocation fails. */
vsie_status vsie_set_tuning(vsie_handle* h, const vsie_tuning* tuning);

/* The precision-32 vsie_apply_batched of nop operators at once, operator p applied to its
 * own block d_x[p] -> d_y[p] (each n x nrhs): the persistent tensor-core launch of each
 * source class covers the items of up to 16 operators, so that several frequencies (or
 * materials) on one mesh share one launch and its load balance.  The operators must agree
 * in n and in the far-field source counts of each class (the same mesh; different k0, rho,
 * c are fine) and be distinct.  hs, d_x, d_y: host arrays of nop entries.  Blocking (reads
 * the kernels' timeout flags).  Errors as vsie_apply_batched; VSIE_ERR_ARG on a size
 * mismatch. */
vsie_status vsie_apply_batched_multi(vsie_handle* const* hs, int32_t nop, const void* const* d_x,
                                     void* const* d_y, int32_t nrhs, void* stream);

/* A CUDA-graph plan of vsie_apply_batched_multi for fixed operators and buffers: create
 * runs the apply once (allocating every scratch buffer, results in d_y), then records all
 * its launches by stream capture on a private stream; launch replays the graph on
 * ``stream`` and blocks until done (reads the timeout flags).  The plan holds the device
 * pointers: the buffers and operators must outlive it, and no other call may use the
 * operators while a launch runs.  nodes: number of graph nodes (launches and copies). */
typedef struct vsie_graph vsie_graph;
vsie_status vsie_graph_create_batched(vsie_handle* const* hs, int32_t nop, const void* const* d_x,
                                      void* const* d_y, int32_t nrhs, vsie_graph** out);
vsie_status vsie_graph_launch(vsie_graph* g, void* stream);
vsie_status vsie_graph_nodes(const vsie_graph* g, int64_t* nodes);
void vsie_graph_destroy(vsie_graph* g);

/* x = A^H y (conjugate transpose: the roles of targets and sources swapped in the far
 * sums, the transposed correction, the real mass), same layouts as vsie_apply; precision
 * 32 or 64 (VSIE_ERR_ARG for 48).  Asynchronous; the first call allocates the adjoint
 * records. */
vsie_status vsie_adjoint_apply(vsie_handle* h, const void* d_y, void* d_x, int32_t nrhs,
                               int32_t precision, void* stream);

/* Right-hand side of Eq. (planewave): b_i = exp(i k0 x_i . d_j) for ndir unit directions
 * (host array 3*ndir, normalised by the library); b: device complex128 n x ndir, column
 * j for direction j.  FP64.  Blocking.  VSIE_ERR_ARG on a null pointer, ndir outside
 * 1..65535 or a zero or non-finite direction. */
vsie_status vsie_plane_wave_rhs(vsie_handle* h, const double* h_dirs, int32_t ndir,
                                void* d_b, void* stream);

/* Far-field pattern of the scattered field from Eq. (vsie) used as a representation
 * formula in Omega_0 (Sec. 2.3.1): p_inf(xhat) = (1/4pi) sum_j e^{-ik0 xhat.y_j}
 * (s_j - i k0 xhat.v_j) p_e(j) over the far-field source points.  p: device complex128
 * n x nrhs; dirs: host 3*ndir; out: device complex128 ndir x nrhs.  FP64.  Blocking.
 * VSIE_ERR_ARG on a null pointer, ndir < 1 or nrhs outside 1..65535. */
vsie_status vsie_far_field(vsie_handle* h, const void* d_p, int32_t nrhs,
                           const double* h_dirs, int32_t ndir, void* d_out, void* stream);

typedef struct {
  int32_t mode;             /* 64: FP64 GMRES with the FP64 apply (the paper's solver,
                               Sec. 3.1); 32: FP64 iterative refinement whose residual
                               uses the FP64 apply around inner FP32-apply GMRES       */
  double tol;               /* relative residual ||b - A x|| / ||b|| to reach          */
  int32_t max_iters;        /* total GMRES iterations (all inner solves)               */
  int32_t restart;          /* Krylov basis size; 0 = max_iters (no restart)           */
  double inner_tol;         /* mode 32: relative tolerance of each inner solve         */
  int32_t max_refinements;  /* mode 32: outer refinement steps                         */
  int32_t adjoint;          /* nonzero: solve A^H x = b (adjoint state of a gradient)   */
  int32_t initial_guess;    /* vsie_solve: nonzero = x holds a starting iterate on entry
                               (resume from a saved x_k: the first residual b - A x is
                               formed with the FP64-accuracy apply); 0 = start from x = 0.
                               Must be 0 for vsie_solve_batched                        */
} vsie_solve_opts;

typedef struct {
  int32_t iterations;       /* total GMRES iterations                                  */
  int32_t refinements;      /* outer steps (mode 32)                                   */
  double rel_residual;      /* final ||b - A x|| / ||b|| with the FP64 apply           */
  int32_t fp64_applies;     /* number of FP64 operator applications                    */
  int32_t fp32_applies;     /* number of FP32 operator applications                    */
} vsie_solve_info;

/* Solve A x = b for one right-hand side from x0 = 0 (GMRES, no preconditioner, as in
 * Sec. 3.1), or from the iterate held in x when opts->initial_guess is set.  b, x: device
 * complex128 (n), caller-owned; the workspace ((basis + 4) x n complex128) is allocated
 * and freed by the call.  Blocking (reads residual norms on the host).  Returns
 * VSIE_ERR_NOT_CONVERGED (x still written, info filled) when the limits are hit,
 * VSIE_ERR_NAN on a non-finite right-hand side or residual, VSIE_ERR_BREAKDOWN when GMRES
 * stalls with a nonzero residual, VSIE_ERR_ARG on invalid options (a basis above 3000
 * columns included). */
vsie_status vsie_solve(vsie_handle* h, const void* d_b, void* d_x,
                       const vsie_solve_opts* opts, vsie_solve_info* info, void* stream);

/* Solve A x_c = b_c for nrhs right-hand sides at once: b, x device complex128, n x nrhs
 * column-major.  Each column runs its own GMRES from x0 = 0 with the options of vsie_solve
 * (Sec. 3.1: no preconditioner, relative residual tolerance) and its own Krylov basis;
 * every operator application is shared by the block (lockstep Arnoldi steps, CGS2).
 *   mode 32: FP64 iterative refinement whose residuals use the FP64 apply, around inner
 *            cycles with the tensor-core multi-RHS FP32 apply of vsie_apply_batched (the
 *            single-column FP32 apply once fewer than four columns remain active);
 *   mode 64: FP64 GMRES with the FP64 apply, column by column.
 * infos: host array of nrhs entries (per-column counts and final residuals) or NULL.
 * The Krylov basis (restart, else max_iters) is limited to 1000 columns; the device
 * workspace is (basis + 4) x n x nrhs complex128, freed on return.  Adjoint solves are
 * rejected (VSIE_ERR_ARG; use vsie_solve).  Blocking.  Returns VSIE_ERR_NOT_CONVERGED when
 * any column misses the tolerance (every x column is still written). */
vsie_status vsie_solve_batched(vsie_handle* h, const void* d_b, void* d_x, int32_t nrhs,
                               const vsie_solve_opts* opts, vsie_solve_info* infos, void* stream);

/* Adjoint of vsie_far_field: x_e = (1/4pi) sum_{j in e} sum_d e^{+ik0 xhat_d.y_j}
 * (s_j + i k0 xhat_d.v_j) r_d, i.e. x = F^H r for the far-field map F of vsie_far_field
 * (the right-hand side of the adjoint equation of a far-field misfit).  r: device
 * complex128 ndir x nrhs; dirs: host 3*ndir; x: device complex128 n x nrhs.  FP64. */
vsie_status vsie_far_field_adjoint(vsie_handle* h, const void* d_r, int32_t nrhs,
                                   const double* h_dirs, int32_t ndir, void* d_x, void* stream);

/* Scattered field at m points outside the scatterer (Sec. 2, Eq. vsie, where the mass
 * function is 1): p_s(X) = p(X) - p_inc(X) = -sum_e I_e(X) p_e, I(X) the integral part of
 * the operator row at X -- the far rule over all far-field source points, with the near
 * rules of the create-time radii (four-point tetrahedron rule; the solid-angle split of the
 * double layer) for elements whose centroids lie within those radii of X.  X must lie
 * outside every tetrahedron (no self term is formed; a point inside gets a meaningless
 * value, not an error).  p: device complex128 n x nrhs (the solved collocation values);
 * points: host 3 m doubles (x, y, z per point, finite); out: device complex128 m x nrhs.
 * precision 32 (FP32 far sums), 48 (double-float) or 64.  Allocates temporaries (the
 * points and their near rows) and blocks until done.  VSIE_ERR_ARG on a bad argument. */
vsie_status vsie_scattered_field(vsie_handle* h, const void* d_p, int32_t nrhs, const double* h_points,
                                 int64_t m, int32_t precision, void* d_out, void* stream);

/* Density gradient of an element-wise density, the least-squares reading: for every
 * tetrahedron e, g_e minimises sum_f (alpha_f - alpha_e - g . (c_f - c_e))^2 over the
 * tetrahedra f sharing a face with e in the same subdomain (c: centroids); the
 * minimum-norm minimiser when those neighbours span fewer than three directions
 * (singular values below 1e-6 of the largest dropped), 0 without neighbours.  It feeds
 * the adjoint double layer (grad(alpha) of Eq. vsie) through vsie_material.grad_alpha.
 * tet_domain: n_tet subdomain labels or NULL (one subdomain); alpha = rho0/rho - 1
 * (n_tet); grad_alpha: 3 n_tet output (x, y, z per tetrahedron).  Host arrays only, no
 * device work; VSIE_ERR_MESH on an out-of-range vertex index. */
vsie_status vsie_lsq_grad_alpha(const vsie_mesh* mesh, const int8_t* tet_domain, const double* alpha,
                                double* grad_alpha);
/* Its adjoint: grad_alpha = W alpha is linear in alpha; d_alpha = W^T d_grad (the chain rule
 * of a gradient with respect to grad_alpha back to alpha).  d_grad: 3 n_tet, d_alpha: n_tet. */
vsie_status vsie_lsq_grad_alpha_adjoint(const vsie_mesh* mesh, const int8_t* tet_domain, const double* d_grad,
                                        double* d_alpha);

/* Gradient channels of an adjoint state lam (device complex128, n): for every far-field
 * source point y_j (the order of vsie_source_points)
 *   phi_j = sum_i conj(G(x_i, y_j)) lam_i,   psi_j = sum_i conj(grad_x G(x_i, y_j)) lam_i,
 * over all collocation points x_i (terms with x_i = y_j vanish), G = e^{ik0 r}/(4 pi r)
 * (Eq. greens_function), grad_x G = G (i k0 r - 1)(x - y)/r^2.  A source point's pair
 * coefficient is C = -G s + grad_x G . v (Eq. vsie), so sum_i conj(dC/ds) lam_i = -phi_j
 * and sum_i conj(dC/dv) lam_i = psi_j: the far-field parts of the derivative of
 * lam^H A p with respect to the source weights s_j and v_j.  d_phi: device complex128
 * n_far; d_psi: device complex128 3 n_far (x, y, z per point).  precision 32 or 64.
 * Asynchronous; the first call allocates the adjoint buffers. */
vsie_status vsie_gradient_channels(vsie_handle* h, const void* d_lam, int32_t precision, void* d_phi,
                                   void* d_psi, void* stream);

/* The far-field source points in the library's order (volume points with grad(alpha) = 0,
 * interface points, volume points with grad(alpha) != 0): h_xyz 3 n_far doubles (may be
 * NULL), h_owner n_far owning unknowns (may be NULL), h_class n_far class indices 0, 1, 2
 * (may be NULL).  Host arrays, caller-owned; blocking. */
vsie_status vsie_source_points(const vsie_handle* h, double* h_xyz, int32_t* h_owner, int32_t* h_class);

/* Measured issue rates of the SM pipes that bound the far-field sums (the paper reports
 * no timings and has no counterpart; this is roofline evidence for the ALU-bound
 * kernels).  On the current device, each of five probe kernels runs independent
 * dependency chains of one instruction in one full wave of blocks.  per_clk_per_sm[5]
 * receives the median over SMs of the operations completed per SM clock (clock64 spans)
 * for: MUFU rsqrt, MUFU sin, scalar FP32 FMA, paired FP32x2 FMA (counted as two FMAs),
 * FP64 FMA.  sm_mhz (may be NULL) receives the SM clock implied by the longest span and
 * the launch's event time.  Allocates and frees a small device buffer; about 0.1 s;
 * blocking.  Errors: VSIE_ERR_ARG (null output), VSIE_ERR_CUDA. */
vsie_status vsie_pipe_probe(double* per_clk_per_sm, double* sm_mhz, void* stream);

/* Thread-local description of the last error ("" if none). */
const char* vsie_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* VSIE_H */
