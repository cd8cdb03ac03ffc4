/*
 * h2bem: boundary double-layer operator of the Fredkin-Koehler FEM/BEM method
 * with H2-matrix compression, on one NVIDIA GB300 (sm_103a).
 *
 * Computes u2|Gamma = M u1|Gamma (arXiv:1811.05731, Eq. (denseMat)) with
 *   M = K + D,
 *   K_ij = (1/4pi) oint phi_j(y) n_y.(xi_i - y)/|xi_i - y|^3 dS_y
 *          (collocation at the nodes xi_i, linear nodal basis phi_j on a flat
 *          triangle mesh, Eq. (matrix_definition); entries by Lindholm's
 *          closed form),
 *   D_ii = Psi(xi_i)/(4 pi) - 1, Psi the interior solid angle (Eq. (mainInt)),
 * where K is compressed as an H2 matrix (Section "H2-Matrix Compression"):
 * a geometric cluster tree, eta-admissible blocks K|t x s ~ V_t S_ts W_s^T
 * with tensor Chebyshev interpolation of order m (k = m^3 coefficients per
 * cluster), nested bases through transfer matrices E_t, and exact FP64 near
 * blocks.  The sign convention of the double-layer term is the one under
 * which a constant u1 gives u2 = -u1 (M 1 = -1).
 *
 * Conventions for every entry point:
 *  - Return value: H2_OK (0) or a negative h2_status; no exception crosses
 *    this interface.  h2_error_string() names a code.
 *  - Streams: `cuda_stream` is a cudaStream_t (NULL = legacy default stream).
 *    Work is stream-ordered; h2_matvec returns before the GPU finishes when
 *    given device buffers.
 *  - Ownership: handles are created by the library and released with
 *    h2_free.  Mesh arrays are copied.  Vector buffers stay owned by the
 *    caller.  An operator keeps its geometry alive until both are freed.
 *  - Thread safety: calls on one handle must not overlap (one workspace per
 *    operator).
 */
#ifndef H2BEM_H
#define H2BEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct h2_handle h2_handle;   /* opaque: a geometry or an operator */

typedef enum {
    H2_OK = 0,
    H2_ERR_INVALID_ARG = -1,          /* null pointer, size out of range, bad parameter */
    H2_ERR_MESH_OPEN = -2,            /* an edge is not shared by exactly two triangles */
    H2_ERR_MESH_ORIENTATION = -3,     /* inconsistent orientation or enclosed volume <= 0 */
    H2_ERR_DEGENERATE_TRIANGLE = -4,  /* zero-area triangle or repeated corner */
    H2_ERR_OOM = -5,                  /* device or host allocation failed */
    H2_ERR_CUDA = -6,                 /* a CUDA runtime call failed */
    H2_ERR_TIMEOUT = -7,              /* a bounded device-side wait gave up */
    H2_ERR_RHS_EXCEEDS_MAX = -8,      /* r > h2_params.max_rhs (h2_matvec_noalloc: its own limit) */
    H2_ERR_WRONG_HANDLE = -9,         /* geometry given where an operator is needed, or vice versa */
    H2_ERR_SCRATCH_LIMIT = -10        /* h2_matvec_noalloc: problem larger than its fixed scratch */
} h2_status;

/* Storage/arithmetic precision of the far field (transfer, coupling and leaf
 * bases).  Near blocks, the solid-angle diagonal, the geometry and the final
 * per-node sum are FP64 in every mode (the near field's arithmetic has one
 * FP64-equivalent alternative, h2_params.near_field).
 *  H2_FP64:   everything FP64 (CUDA cores).
 *  H2_FP32:   far-field matrices and vectors (x-hat, y-hat) in FP32, FP32
 *             products with FP32 accumulation on the CUDA cores.
 *  H2_TF32X3: as H2_FP32, but the coupling and transfer products run on the
 *             tensor cores (tcgen05) as three TF32 products per term
 *             (hi*hi + hi*lo + lo*hi, hi = the nearest TF32 value, lo = the
 *             nearest TF32 value of the remainder), FP32 accumulation.
 *  H2_BF16X3: coupling matrices stored as BF16 pairs hi + lo (hi = bf16(a),
 *             lo = bf16(a - hi), 4 bytes per entry, |a - hi - lo| <= 2^-18 |a|)
 *             and multiplied on the tensor cores with the FP32 vectors split
 *             into three BF16 words x = xh + xm + xl (exact), as
 *             hi*(xh + xm + xl) + lo*(xh + xm), FP32 accumulation; transfer
 *             matrices and leaf bases FP32 on the CUDA cores (the same 4 bytes
 *             per entry).
 * For products of at most 4 right-hand sides the H2_TF32X3 and H2_BF16X3 tiles
 * are multiplied on the CUDA cores (the same stored values, FP32 products and
 * accumulation), where one tensor-core instruction of so few columns costs as
 * much as one of 128; h2_autotune may choose the tensor cores instead.
 * The reduced forms target a relative error <= 1e-5 against the FP64 form;
 * BF16 hi + lo keeps about 17 significant bits of each coupling entry, which
 * the far-field sums amplify to 5e-6 .. 1.3e-5 on the benchmark meshes. */
typedef enum { H2_FP64 = 0, H2_FP32 = 1, H2_TF32X3 = 2, H2_BF16X3 = 3 } h2_precision;

typedef struct {
    int32_t m;              /* Chebyshev points per axis, 1..5 (k = m^3 <= 125)       */
    int32_t leaf;           /* maximum nodes per leaf cluster, 1..128                 */
    double eta;             /* admissibility: max(diam) <= eta * dist                 */
    double box_inflation;   /* rho: every box side >= rho * longest side (0.25)       */
    int32_t precision;      /* h2_precision                                           */
    int32_t max_rhs;        /* largest r accepted by h2_matvec (workspace size), >= 1 */
    int32_t schedule;       /* h2_schedule: how one h2_matvec is launched              */
    int32_t autotune;       /* 1: h2_assemble ends with h2_autotune(op, max_rhs)       */
    int32_t coupling;       /* h2_coupling: stored S_ts (default) or evaluated        */
    int32_t near_field;     /* h2_near_field: near-field arithmetic (default FP64)     */
    double recompress_eps;  /* 0 (default): interpolation bases of rank k = m^3; in
                               (0, 1): algebraic recompression of the far field with
                               relative threshold eps (see h2_assemble)              */
} h2_params;

/* H2_COUPLING_STORED (default): the coupling matrices S_ts are assembled and
 *   stored in the operator's precision and streamed by every product.
 * H2_COUPLING_ON_THE_FLY (H2_FP32 operators only): every product evaluates
 *   S_ts(nu, mu) = 1 / (4 pi |x^t_nu - x^s_mu|) (Section "H2-Matrix
 *   Compression": the coupling matrices are the kernel at the interpolation
 *   nodes) in FP32 from the Chebyshev nodes, stored per block relative to the
 *   target box's centre so that the difference keeps its digits; the coupling
 *   matrices, the largest part of the far field, are neither stored nor
 *   streamed. */
typedef enum { H2_COUPLING_STORED = 0, H2_COUPLING_ON_THE_FLY = 1 } h2_coupling;

/* Arithmetic of the near-field product y|_t += sum_s N_ts x|_s (the exact
 * Lindholm blocks of the inadmissible leaf pairs, Section "H2-Matrix
 * Compression": only the admissible blocks are approximated).
 * H2_NEAR_FP64 (default): FP64 entries, FP64 products and sums.
 * H2_NEAR_F32PAIR (H2_FP32 and H2_BF16X3 operators with max_rhs > 8): the
 *   products that run in the split form (more than 8 right-hand sides, see
 *   h2_params.max_rhs) carry every near-field entry and input value as an
 *   unevaluated pair of FP32 numbers hi + lo (hi = fp32(v), lo = fp32(v - hi):
 *   48 significant bits) and multiply them with error-free transformations on
 *   the FP32 pipe, which GB300 runs at 64 times its FP64 rate: the exact
 *   product hi_a*hi_x as a rounded product and its FMA-computed error
 *   (Dekker 1971), the cross terms hi_a*lo_x + lo_a*hi_x, and a running sum
 *   kept as a rounded sum plus its TwoSum error (Knuth 1969).  Each leaf's
 *   result is converted to FP64 once and added to the FP64 output.  The
 *   error of a row of n terms stays below n * 2^-48 times the sum of the
 *   magnitudes of its terms (the low word's own rounding grows with the row;
 *   about 6e-13 for 1000 terms), within the FP64 path's 1e-8 and far inside
 *   the reduced forms' 1e-5.  A paired copy of the near blocks is kept beside
 *   the FP64 ones (the same bytes again), which products with at most 8
 *   right-hand sides still use.  An operator without the split form (a leaf
 *   above 64 rows, or the level-wise schedule without h2_params.autotune)
 *   keeps the FP64 near field for every product; h2_stats reports
 *   bytes_near_pair = 0 then. */
typedef enum { H2_NEAR_FP64 = 0, H2_NEAR_F32PAIR = 1 } h2_near_field;

/* H2_SCHEDULE_FLOW (default): one persistent kernel after the input gather;
 *   its CTAs take the product's segments in a dependency order and wait
 *   (bounded) for the cluster vectors they read.
 * H2_SCHEDULE_LEVELS: one kernel per pass (upward leaf projection, each
 *   upward level, coupling, each downward level, near field, leaf expansion). */
typedef enum { H2_SCHEDULE_FLOW = 0, H2_SCHEDULE_LEVELS = 1 } h2_schedule;

/* Fills `p` with the defaults: m = 4, leaf = 64, eta = 2, rho = 0.25, FP64, max_rhs = 1,
 * flow schedule. */
void h2_default_params(h2_params* p);

/* Build a geometry handle from a closed, outward-oriented triangle mesh
 * (Section "Discretization": nodes xi_i, piecewise linear nodal basis).
 *   xyz: host, n_vertices x 3 doubles, row-major.
 *   tri: host, n_triangles x 3 int32 node indices (0-based), counter-clockwise
 *        seen from outside.
 * Validates closedness, orientation and non-degeneracy (error codes above),
 * copies the mesh to the device and computes the interior solid angle Psi at
 * every node (Eq. (mainInt)).  Returns the handle in *out_geom. */
int h2_build_geometry(const double* xyz, int64_t n_vertices, const int32_t* tri,
                      int64_t n_triangles, void* cuda_stream, h2_handle** out_geom);

/* Assemble the H2 operator on the device (Section "H2-Matrix Compression"):
 * cluster tree, block partition, leaf bases V_t and W_t, transfer matrices
 * E_t, coupling matrices S_ts and FP64 Lindholm near blocks with the
 * solid-angle diagonal.  `p` may be NULL (defaults).  Synchronous.
 * With p->recompress_eps = eps > 0 the far field is then compressed
 * algebraically on the device, in FP64, before it is stored in the operator's
 * precision (the paper's recompression of the cluster bases after their
 * construction, Section "H2-Matrix Compression"; the steps of Boerm's
 * algorithms for nested bases): the row and column bases are orthogonalised
 * (QR, leaves to root), their total weights formed (root to leaves) and
 * truncated to the left singular vectors whose singular values exceed eps
 * times the largest (leaves to root), which gives every cluster its own rank
 * <= k and new couplings B_t S_ts B_s^T.  The product's error against the
 * interpolation operator is about 0.02 eps on the benchmark meshes; the
 * streamed bytes fall with the ranks (h2_stats).  Needs stored couplings
 * (H2_COUPLING_STORED); H2_ERR_INVALID_ARG for eps < 0 or eps >= 1.  The
 * recompression uses FP64 scratch of about the interpolation far field's
 * FP64 size twice over, released before the call returns. */
int h2_assemble(const h2_handle* geom, const h2_params* p, h2_handle** out_op);

/* u2 = M u1 for r right-hand sides (Eq. (denseMat)).
 *   u1, u2: r x N doubles, row-major (right-hand side c at offset c*N), node
 *           order of the input mesh.  Either both device pointers or both
 *           host pointers; with host pointers the call copies in and out on
 *           `cuda_stream` and returns after the result is in u2.
 *   1 <= r <= max_rhs.  u1 and u2 must not overlap.  u2 is overwritten.
 * The work is ordered on `cuda_stream`; FP32 and BF16 hi+lo operators with
 * r > 8 also run the near field on a stream of the operator, joined to
 * `cuda_stream` by events before the call's last launch (the result is
 * complete when `cuda_stream` reaches that point, as for every call). */
int h2_matvec(h2_handle* op, const double* u1, double* u2, int32_t r, void* cuda_stream);

/* u2_i = M_i u1_i for several operators at once (several meshes, e.g. of
 * uneven size): after one input gather per operator, ONE persistent kernel
 * launch runs the products of all of them, their segments scheduled together
 * (Eq. (denseMat) for each mesh).
 *   ops:    n_ops distinct operator handles, 1 <= n_ops <= 16, on one device.
 *   u1, u2: n_ops DEVICE pointers; u1[i], u2[i] are r[i] x N_i doubles,
 *           row-major, mesh node order; they must not overlap.
 *   r:      n_ops right-hand-side counts, 1 <= r[i] <= max_rhs of ops[i].
 * Asynchronous on `cuda_stream`.  The first call for a set of operators
 * builds and caches the combined schedule (host work and device arrays,
 * released when one of the operators is freed).  A bounded device-side wait
 * that gives up is reported by h2_device_status(ops[0]).  Calls involving
 * the same operator must not overlap. */
int h2_matvec_batched(h2_handle* const* ops, int32_t n_ops, const double* const* u1, double* const* u2,
                      const int32_t* r, void* cuda_stream);

/* u2 = M u1 like h2_matvec, for callers that cannot allocate device memory
 * while they apply the operator (for example a time-stepping loop that
 * reserved all device memory in advance, or an application whose device
 * memory belongs to its own pool allocator).  The paper has no counterpart:
 * this is a property of the library, not of the method.
 *   u1, u2: DEVICE pointers only, r x N doubles as in h2_matvec.
 *   r:      1 <= r <= 8 for an operator assembled with max_rhs <= 8, else
 *           1 <= r <= 32 (either may exceed max_rhs); a larger r returns
 *           H2_ERR_RHS_EXCEEDS_MAX without launching anything.
 * The calling thread's current device must be the operator's device
 * (H2_ERR_INVALID_ARG otherwise).  Asynchronous on `cuda_stream`.
 * The workspace is a fixed array of 4,194,304 doubles (32 MiB) inside the
 * library, present on every GPU that loads it until the process exits.
 * It must hold W = rows x r doubles, rows = (the mesh nodes, each leaf
 * cluster's count rounded up to a multiple of 4) + 2 x n_clusters x k4 + 4
 * with k4 = m^3 rounded up to a multiple of 4, and for reduced-precision
 * operators W more floats after a 256-byte boundary; larger problems get
 * H2_ERR_SCRATCH_LIMIT without anything being launched.  No cudaMalloc, cudaFree
 * or other allocating routine is called.  The first call on a device looks up
 * the array's device address (and loads the library's kernels on that
 * device); make it before any stream capture.  Every call shares the array:
 * calls whose executions overlap on the GPU race and give wrong results. */
int h2_matvec_noalloc(h2_handle* op, const double* u1, double* u2, int32_t r, void* cuda_stream);

/* Launch configuration of an operator's product, as chosen by h2_autotune. */
typedef struct {
    int32_t schedule;       /* h2_schedule                                            */
    int32_t stages;         /* shared-memory stages of the segment kernel             */
    int32_t ctas_per_sm;    /* resident CTAs per SM                                    */
    int32_t n_candidates;   /* configurations timed                                   */
    double ms_best;         /* mean time of one product in the chosen configuration   */
    double ms_default;      /* the same with the configuration h2_assemble chose      */
} h2_tuning_t;

/* Autotuner of the product's launch configuration (not part of the method: a
 * property of this implementation).  Times, with CUDA events on `cuda_stream`
 * and products of r right-hand sides on zero-filled scratch vectors, every
 * combination of the schedule (the single dataflow launch or one launch per
 * pass), 2..4 shared-memory stages and 1..max resident CTAs per SM that fits,
 * and, where they apply, the split form (r > 8, FP32 and BF16 hi+lo: the FP64
 * near field in its own launch beside the rest) and the pipe of 3xTF32 / BF16
 * hi+lo tiles at r <= 4 (CUDA cores or tensor cores); keeps the fastest for
 * later h2_matvec calls (the dataflow ticket order is rebuilt for its CTA
 * count) and reports it in *out (may be NULL; `schedule` reports the split
 * form as H2_SCHEDULE_FLOW).  The matrices and their layout do not change; the
 * results change only by rounding.  Allocates and frees its scratch vectors;
 * synchronous.  1 <= r <= max_rhs. */
int h2_autotune(h2_handle* op, int32_t r, void* cuda_stream, h2_tuning_t* out);

/* Counts and sizes of an operator (Section "Results", "Data compression":
 * storage of the compressed operator and the compression ratio
 * r = 1 - size(compressed) / size(dense)). */
typedef struct {
    int64_t n_vertices, n_triangles;
    int32_t n_clusters, n_levels, n_leaves, k;
    int64_t n_far_blocks, n_near_blocks;
    int64_t near_entries;          /* FP64 near-field entries (incl. the diagonal)      */
    int64_t far_coefficients;      /* coupling entries: n_far_blocks * k^2              */
    int64_t basis_coefficients;    /* stored V, W and transfer entries                  */
    int64_t bytes_far;             /* device bytes of S, V, W and the transfers         */
    int64_t bytes_near;            /* device bytes of the near blocks                   */
    int64_t bytes_streamed;        /* matrix bytes one matvec reads (each exactly once) */
    int64_t macs_per_rhs;          /* multiply-adds of one matvec per right-hand side   */
    double compression_ratio;      /* 1 - (far + near bytes) / (8 N^2)                  */
    double assemble_seconds;
    int32_t precision, max_rhs;
    int32_t n_launches_matvec;     /* kernel launches per h2_matvec                     */
    int32_t n_passes;              /* block-sparse passes per h2_matvec                 */
    int64_t bytes_near_pair;       /* device bytes of the paired near-field copy (0
                                      unless h2_params.near_field = H2_NEAR_F32PAIR)   */
    int32_t near_field, coupling;  /* h2_near_field and h2_coupling of the operator     */
    double recompress_eps;         /* h2_params.recompress_eps of the operator           */
    double mean_rank_row;          /* mean rank of the row bases the product uses (k
                                      without recompression)                            */
    double mean_rank_col;          /* the same for the column bases                     */
    int32_t max_rank;              /* the largest rank of a cluster basis               */
} h2_stats_t;

int h2_stats(const h2_handle* op, h2_stats_t* out);

/* Copy the cluster tree out (host arrays; sizes from h2_stats):
 *   perm[N]: node at tree position q; start/size/parent/child0/child1/level
 *   [n_clusters] (child = -1 at leaves; clusters numbered level by level);
 *   box[6*n_clusters]: lo xyz, hi xyz of the interpolation box. */
int h2_get_tree(const h2_handle* op, int32_t* perm, int32_t* start, int32_t* size,
                int32_t* parent, int32_t* child0, int32_t* child1, int32_t* level,
                double* box);

/* Copy the block partition out (host arrays of n_far_blocks / n_near_blocks). */
int h2_get_blocks(const h2_handle* op, int32_t* far_t, int32_t* far_s, int32_t* near_t,
                  int32_t* near_s);

/* Copy Psi (N doubles, mesh node order) of a geometry or operator to host memory. */
int h2_get_psi(const h2_handle* h, double* psi);

/* Synchronises the device and reports whether any h2_matvec on `op` since
 * the last call gave up a bounded device-side wait (H2_ERR_TIMEOUT; the
 * result of that product is then undefined).  Clears the flag.  While the
 * flag is set, later dataflow products on `op` stop at their first wait for
 * another CTA's output (their results are undefined too): read the status
 * after a product whose result matters. */
int h2_device_status(h2_handle* op);

/* Failure-detection test hook (not part of the method).  enable = 1 makes
 * the dataflow product of `op` wait for one more signal of a region than its
 * producers ever send, so that the waiting CTA's bounded wait (1 s) runs out:
 * the product stops early, leaves u2 undefined and h2_device_status(op)
 * returns H2_ERR_TIMEOUT; the CUDA context stays usable.  enable = 0
 * restores the operator.  Only for operators with the dataflow schedule;
 * synchronises the device. */
int h2_fault_inject_stall(h2_handle* op, int32_t enable);

/* Per-pass timing (a measurement aid, not needed for computing).  While
 * enabled, every h2_matvec on `op` records CUDA events on its stream before
 * and after each kernel launch.  Enabling or disabling drops what was
 * recorded so far. */
int h2_profile_enable(h2_handle* op, int32_t enable);

/* Synchronises on the recorded events and returns, per kernel launch of one
 * h2_matvec in launch order (the input gather, then one entry per pass, or
 * one entry for the single flow kernel; the split form: gather, near field,
 * far-field flow kernel, joining addition, per product of at most 16
 * right-hand sides), the kind (0 gather, 1 upward leaf projection, 2 upward
 * transfer, 3 coupling, 4 downward transfer, 5 near field, 6 leaf expansion,
 * 7 the whole flow kernel, 8 the split form's near field, 9 its far-field
 * flow kernel, 10 its addition), the total milliseconds over all recorded
 * calls (each launch timed by events recorded before and after it on the
 * stream it runs on), the matrix bytes and the multiply-adds (per
 * right-hand side) of one launch, and its grid size.  Arrays hold
 * `capacity` entries (any may be NULL); *n_entries is the number of launches
 * per call and *n_calls the number of recorded calls.  Clears the recorded
 * events. */
int h2_profile_read(h2_handle* op, int32_t capacity, int32_t* kind, double* ms_total,
                    int64_t* bytes, int64_t* macs, int32_t* grid, int32_t* n_calls,
                    int32_t* n_entries);

/* Host-only check of the execution plan (no device work, usable without a
 * GPU): builds, for a mesh and parameters, the cluster tree, the block
 * partition (Section "H2-Matrix Compression"), the passes of the product and
 * the dataflow ticket order (with and without the near field, and merged
 * with a second copy of itself as a batched launch merges operators) exactly
 * as h2_assemble and h2_matvec_batched do, with the ticket order simulated for `workers` concurrent
 * CTAs, and checks the invariants the product kernels rely on, independently
 * of the code that built them: every chunk a legal bulk copy (16-byte aligned
 * source and size, within one stage, input rows on 4-row boundaries, one
 * piece type per chunk, one accumulator kind per segment); the ticket order
 * topological (every producer of a region a segment waits for holds an
 * earlier ticket, so persistent CTAs cannot deadlock); every region's
 * expected signal count equal to the writer signals of its producers.
 * `violations` counts the failed checks (0 for a sound plan).  The mesh is
 * validated as by h2_build_geometry (same error codes); `params` as by
 * h2_assemble (NULL: defaults).  Host arrays only. */
typedef struct {
    int32_t n_clusters, n_levels;
    int64_t n_far_blocks, n_near_blocks;
    int64_t n_segments, n_chunks;     /* dataflow form with the near field        */
    int64_t n_split_segments;         /* without the near field (-1: no order)     */
    int32_t n_regions, violations;
    int64_t bytes_streamed;           /* matrix bytes one product reads            */
    double makespan_us;               /* simulated makespan of the ticket order    */
    double split_makespan_us;         /* the same without the near field (-1)      */
} h2_plan_report_t;

int h2_plan_check(const double* xyz, int64_t n_vertices, const int32_t* tri, int64_t n_triangles,
                  const h2_params* params, int32_t workers, h2_plan_report_t* out);

/* ---- The finite-element half of the field evaluation ----
 * Section "Basic Equations" (Fredkin-Koehler): the magnetostatic potential
 * u = u1 + u2 of a body with magnetisation M, on a tetrahedral mesh with
 * linear (P1) elements:
 *   u1: Poisson problem with Neumann data M.n (Eqs. u1Poiss, u1Neumann),
 *       weak form int grad u1 . grad v = int M . grad v for all P1 v, made
 *       unique by a zero mean (lumped volume weights);
 *   u2: harmonic, boundary values from the boundary integral equation
 *       (Eq. mainInt) = the operator's product with u1 on the boundary
 *       (h2_matvec), interior values from the P1 Dirichlet problem;
 *   e_d / K_d = (1/V) int M . grad(u1 + u2) dV, K_d = mu0 Ms^2 / 2 (Section
 *       "Magnetostatic field and energy"; for a uniform unit M the
 *       demagnetising factor along M).
 * Both linear systems are solved on the device by conjugate gradients
 * preconditioned with the stiffness matrix's diagonal (FP64). */

/* Build a tetrahedral-mesh handle (host arrays, copied):
 *   xyz:  n_vertices x 3 doubles;  tets: n_tets x 4 int32 vertex indices,
 *         each tetrahedron of positive volume (H2_ERR_MESH_ORIENTATION
 *         otherwise);
 *   surf_nodes: the volume index of every node of the boundary surface, in
 *         the node order of the surface mesh the operator was built on
 *         (h2_build_geometry of the boundary faces, outward).
 * Assembles the P1 stiffness matrix (CSR) and the element volumes and
 * gradients on the current device.  Synchronous. */
int h2_fem_create(const double* xyz, int64_t n_vertices, const int32_t* tets, int64_t n_tets,
                  const int32_t* surf_nodes, int64_t n_surf, h2_handle** out_fem);

typedef struct {
    int32_t iters_u1, iters_u2;   /* conjugate-gradient iterations of the two solves       */
    double resid_u1, resid_u2;    /* their final relative residuals |r| / |b|              */
    double energy;                /* e_d / K_d                                             */
    double volume;                /* the body's volume (sum of the tetrahedra)             */
} h2_fem_report_t;

/* u1, u2 and the energy for the magnetisation M (DEVICE, n_tets x 3 doubles,
 * one vector per tetrahedron).  u1, u2: DEVICE, n_vertices doubles each,
 * overwritten.  `op`: an operator on the boundary surface (its N = n_surf).
 * The solves stop at |r| <= tol |b| or after max_iter iterations each (see
 * the report); the residual is checked every 8 iterations (they run as a
 * CUDA graph captured on a stream of the library's own and launched on
 * `cuda_stream`), so a solve may take up to 7 iterations past the one that
 * met tol.  Allocates scratch for the call; synchronous on `cuda_stream`,
 * which must not itself be capturing. */
int h2_fem_solve(h2_handle* fem, h2_handle* op, const double* M, double* u1, double* u2, double tol,
                 int32_t max_iter, void* cuda_stream, h2_fem_report_t* out);

/* Release a geometry, operator or tetrahedral-mesh handle; NULL is a no-op.
 * Releasing a handle twice is undefined. */
int h2_free(h2_handle* h);

/* Static string naming a status code. */
const char* h2_error_string(int code);

/* Text of the last CUDA error seen by this thread ("" if none). */
const char* h2_last_error_message(void);

#ifdef __cplusplus
}
#endif

#endif /* H2BEM_H */
