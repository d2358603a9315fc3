/*
 * vtm.h — C ABI of the GB300 (sm_103a) Virtual Transmission Method library.
 *
 * The library solves A x = b for a sparse symmetric positive-definite A (§1, §3 eq. 3.1: A is
 * viewed as an electric graph with vertex weights a_ii, edge weights a_ij, current sources b_i
 * and potentials x_i).  It splits the graph by Electric Vertex Splitting (§4, steps 1-4), joins
 * every pair of facing copies with a virtual transmission line of impedance Z (§5), factors each
 * subsystem's local SPD matrix once (eq. 5.8) and iterates Table 1: every sweep solves all
 * subsystems with the incident waves of the previous sweep and exchanges the outgoing waves
 * between twins (Neighbor-To-Neighbor, §1, Table 1 steps 3-5).
 *
 * Conventions for every entry point:
 *  - Return value: VTM_OK (0) or a vtm_status error code; the thread-local message of the last
 *    failure is returned by vtm_last_error().  No entry point aborts or throws.
 *  - Ownership: the caller owns every array it passes; the library copies what it keeps.
 *    Opaque handles are released with the matching *_destroy call (NULL is accepted).
 *  - Host pointers are marked "host", device pointers "device" (memory of the current CUDA
 *    device, e.g. a torch tensor's data_ptr()).  Pointers marked "host or device" are
 *    classified with cudaPointerGetAttributes.
 *  - Right-hand sides and solutions are column-major n x nrhs with leading dimension ld >= n:
 *    element (i, r) is at p[i + r*ld].
 *  - Streams: `cuda_stream` is a cudaStream_t (NULL = legacy default stream).  Work is queued on
 *    it; calls that return host data synchronise it.
 */
#ifndef VTM_H
#define VTM_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define VTM_VERSION_MAJOR 0
#define VTM_VERSION_MINOR 1

typedef enum vtm_status {
  VTM_OK = 0,
  VTM_ERR_INVALID = 1,        /* bad argument, size or handle                                   */
  VTM_ERR_NOT_SYMMETRIC = 2,  /* A is not symmetric (§3 requires a_ij = a_ji)                   */
  VTM_ERR_NOT_CONFORMAL = 3,  /* a boundary vertex is not weakly diagonally dominant, so the
                                 equal-share split cannot make the pieces SNND (Cor. 4.1)        */
  VTM_ERR_NOT_SPD = 4,        /* a local matrix of eq. 5.8 had a non-positive Cholesky pivot     */
  VTM_ERR_NOT_CONVERGED = 5,  /* maxit sweeps without reaching rtol                              */
  VTM_ERR_DIVERGED = 6,       /* residual became NaN/Inf or grew without bound                   */
  VTM_ERR_TIMEOUT = 7,        /* a bounded device wait ran out (kernel returned early)           */
  VTM_ERR_CUDA = 8,           /* a CUDA runtime call failed                                      */
  VTM_ERR_OOM = 9             /* device or host allocation failed                                */
} vtm_status;

/* Symmetric sparse matrix, full storage (both triangles), host memory.
 * rowptr: n+1 int64; col: nnz int32 (sorted ascending within a row, no duplicates);
 * val: nnz float64.  Must be symmetric with a positive diagonal. */
typedef struct vtm_csr {
  int64_t n;
  int64_t nnz;
  const int64_t* rowptr;
  const int32_t* col;
  const double* val;
} vtm_csr;

/* ----------------------------------------------------------------------------------------------
 * Partition (Electric Vertex Splitting, §4)
 * --------------------------------------------------------------------------------------------*/

enum vtm_partition_kind {
  /* Grid cut into blocks that SHARE their cut lines/planes (§9's testbenches are 2D grids cut into
   * blocks; Fig. 7 gives the 2- and 3-level splits).  Vertex id = x + dims[0]*(y + dims[1]*z).
   * Along an axis of extent m with spacing s the cut coordinates are s, 2s, ...; block q covers
   * [q*s, min((q+1)*s, m-1)].  Subgraph id of block (qx,qy,qz) = qx + Bx*(qy + By*qz).
   * Lines: hypercube rule — the copies of a vertex in two blocks that differ along exactly one
   * axis are joined by one line (1 line per copy on a face, 2 on an edge line, 3 at a corner). */
  VTM_PART_GRID = 1,
  /* Owner sets given per vertex; the lines are given explicitly. */
  VTM_PART_OWNERS = 2,
  /* A complete split given explicitly: copies, local matrices Ã_j, source shares and lines
   * (any conformal scheme, e.g. the uneven shares of Example 4.1). */
  VTM_PART_EXPLICIT = 3,
  /* Finite elements split by elements (§4: "do the partitioning on the physical level"): every
   * element belongs to one subgraph, Ã_j is the sum of its elements' matrices (each SPSD, so every
   * piece is SNND, Cor. 4.1, and the pieces sum to A exactly up to rounding); b_i is shared as
   * b_i/|O(i)|.  Elements go to subgraphs by elem_piece, or, when elem_piece is NULL, by recursive
   * coordinate bisection of elem_coords into npieces parts (split the element set at position
   * floor(|E| * floor(p/2) / p) of its order by (coordinate, element id) along the axis of largest
   * extent; the first part recursively gets ids base..base+floor(p/2)-1).  Copies inside a
   * subgraph are in reverse Cuthill-McKee order (start: a minimum-degree node, smallest id on ties;
   * neighbours by increasing degree, then id).  Lines: the copies of vertex i in subgraphs p and q
   * are joined when an element edge through i has elements of both p and q around it. */
  VTM_PART_ELEMENTS = 4,
  /* General conformal split of App. 1 (Lemma A1.1, Thm 4.2) for any SPD A, including matrices
   * that are not diagonally dominant (where step 3's rule returns VTM_ERR_NOT_CONFORMAL).  home[i]
   * in [0, npieces) is the home subgraph of vertex i (every id needs one vertex).  The id range
   * [lo, hi) of a subgraph is halved at mid = (lo + hi) / 2 (recursive bisection, N - 1 splits):
   * alpha = copies with home < mid, the boundary B = alpha copies joined to a beta copy by the
   * subgraph's matrix M, I_a = alpha \ B, I_b = beta.  Completing the square over each interior,
   * T_a = M_Ba M_aa^{-1} M_aB, T_b = M_Bb M_bb^{-1} M_bB, S = M_BB - T_a - T_b (SPD); alpha gets
   * T_a + lambda S on B, beta gets T_b + (1 - lambda) S on new copies of B (both SPD, and they sum
   * to M).  A new copy's home is the smallest home among its beta neighbours; source shares are
   * divided lambda : 1 - lambda; one line joins the two copies.  Copies inside a subgraph are in
   * ascending vertex order.  The boundary blocks are dense and the construction is dense (O(n^3)
   * work, O(n^2) memory): n <= 8192, else VTM_ERR_INVALID; VTM_ERR_NOT_SPD if A is not SPD. */
  VTM_PART_CONFORMAL = 5
};

/* Split rule of GRID and OWNERS (§4 step 3; the paper leaves the shares open, this is the
 * library's rule): edge (i,j) goes to every subgraph in O(i)∩O(j) with weight a_ij/|O(i)∩O(j)|;
 * the copy of a boundary vertex i gets a_ii^(c) = sum_{j!=i} |a_ij^(c)| + delta_i/|O(i)| with
 * delta_i = a_ii - sum_{j!=i}|a_ij| (delta_i < -64 eps a_ii => VTM_ERR_NOT_CONFORMAL; rounding-
 * level negatives count as 0); inner vertices keep a_ii; b_i is shared as b_i/|O(i)|.
 * Copies inside a subgraph are ordered by ascending global vertex id. */
typedef struct vtm_partition_spec {
  int32_t kind;             /* vtm_partition_kind */
  /* GRID */
  int32_t dims[3];          /* grid extents; use 1 for unused axes                           */
  int32_t block[3];         /* cut spacing per axis (>= 1)                                   */
  /* OWNERS */
  int32_t npieces;          /* number of subgraphs (OWNERS, EXPLICIT)                        */
  const int64_t* owner_ptr; /* host, n+1: owners of vertex i are owner_piece[owner_ptr[i]..]  */
  const int32_t* owner_piece; /* host, sorted ascending per vertex, values in [0, npieces)    */
  int64_t nlines;           /* OWNERS: lines as (vertex, piece_a, piece_b) triples            */
  const int64_t* line_vertex;
  const int32_t* line_piece_a;
  const int32_t* line_piece_b;
  /* EXPLICIT: C copies numbered piece by piece */
  const int64_t* piece_ptr;   /* host, npieces+1: copies of piece j are piece_ptr[j]..piece_ptr[j+1]-1 */
  const int64_t* copy_vertex; /* host, C: parent vertex of each copy                             */
  const double* copy_share;   /* host, C: b̃_c = copy_share[c] * b[copy_vertex[c]]              */
  const int64_t* local_rowptr;/* host, C+1: row c of Ã (its piece's local matrix)                */
  const int32_t* local_col;   /* host: LOCAL column index within the piece (0-based)             */
  const double* local_val;    /* host                                                            */
  int64_t ncopy_lines;        /* EXPLICIT: lines as pairs of copy ids                            */
  const int64_t* line_copy_a;
  const int64_t* line_copy_b;
  /* ELEMENTS */
  int64_t nelem;              /* number of elements                                              */
  int32_t nodes_per_elem;     /* k (3 for triangles)                                              */
  int64_t nnodes;             /* nodes of the mesh (including eliminated ones)                    */
  const int64_t* elem_nodes;  /* host, nelem x k mesh node ids                                    */
  const double* elem_mats;    /* host, nelem x k x k element matrices (row-major)                 */
  const int64_t* node_unknown;/* host, nnodes: row of A of each node, -1 if eliminated            */
  const int32_t* elem_piece;  /* host, nelem subgraph ids, or NULL for RCB                        */
  const double* elem_coords;  /* host, nelem x coord_dim (RCB)                                    */
  int32_t coord_dim;
  /* CONFORMAL */
  const int32_t* home;        /* host, n home subgraph ids                                        */
  double lambda;              /* share of the boundary Schur complement kept by alpha, (0, 1)     */
} vtm_partition_spec;

typedef struct vtm_partition vtm_partition;

typedef struct vtm_partition_info {
  int64_t n;          /* vertices of A                       */
  int32_t npieces;    /* subgraphs N                         */
  int64_t ncopies;    /* total local unknowns                */
  int64_t nlines;     /* virtual transmission lines          */
  int64_t nboundary;  /* vertices with two or more copies    */
  int64_t max_piece;  /* largest subgraph (local unknowns)   */
} vtm_partition_info;

/* §4 steps 1-4.  A: host CSR (copied).  On success *out owns the split.
 * A is checked first: rowptr must start at 0, end at nnz >= 0 and never decrease (checked for
 * every row before any entry is read), columns in range and strictly ascending, a positive
 * diagonal in every row, and a_ij = a_ji; a bad rowptr is reported before any entry defect, and
 * of several entry defects the one in the lowest row.  Errors: VTM_ERR_INVALID (a malformed A / bad spec / an edge in no common subgraph /
 * a line between copies that do not exist), VTM_ERR_NOT_SYMMETRIC, VTM_ERR_NOT_CONFORMAL,
 * VTM_ERR_OOM (host memory). */
int vtm_partition_evs(const vtm_csr* A, const vtm_partition_spec* spec, vtm_partition** out);
int vtm_partition_get_info(const vtm_partition* p, vtm_partition_info* info);
/* Recursive coordinate bisection used by VTM_PART_ELEMENTS (rule in its comment): coords host
 * n x dim (dim 1..3), out host n subgraph ids in [0, nparts).  Host only. */
int vtm_rcb(const double* coords, int64_t n, int32_t dim, int32_t nparts, int32_t* out);
/* Subgraph j (eq. 4.4): copies' parent vertices (host, n_j int64), shares (host, n_j double) and
 * Ã_j in local CSR (rowptr n_j+1 int64, col int32, val double).  Any output may be NULL; call
 * first with NULL arrays to read *n_j and *nnz_j. */
int vtm_partition_get_piece(const vtm_partition* p, int32_t j, int64_t* n_j, int64_t* nnz_j,
                            int64_t* vertices, double* shares, int64_t* rowptr, int32_t* col,
                            double* val);
/* Lines as (piece_a, local_a, piece_b, local_b) quadruples, host int64 array of 4*nlines. */
int vtm_partition_get_lines(const vtm_partition* p, int64_t* quads);
/* Candidate couplings for coupled lines (§7.2): every pair of lines t < t' of one bundle (both
 * join the same two subgraphs) whose copies are neighbours in both subgraphs, ordered by t, then
 * by the position of the neighbour in t's local row of its side-a subgraph.  pairs: host,
 * 2 x count int64 (t, t'); weights: host, count doubles, |a_ik| of the original matrix for the
 * vertices i, k of the two lines (the coupling rule y_p = gamma |a_ik| follows the local
 * conductance).  Call with NULL arrays to read *count.  Host only. */
int vtm_partition_line_pairs(const vtm_partition* p, int64_t* count, int64_t* pairs, double* weights);
void vtm_partition_destroy(vtm_partition* p);

/* ----------------------------------------------------------------------------------------------
 * Solver setup (Table 1 steps 1-2, eq. 5.8 factored once, §8)
 * --------------------------------------------------------------------------------------------*/

enum vtm_z_mode {
  VTM_Z_UNIFORM = 0,   /* every line has impedance z_uniform (Example 5.1 style)            */
  VTM_Z_EXPLICIT = 1,  /* z_lines[t] per line, in the order of vtm_partition_get_lines      */
  VTM_Z_MATCHED = 2,   /* impedance matching (§7.1): start from z_uniform on every line,
                          compute each end's input impedance (Def. 7.1 with the other lines
                          terminated), set Z_t = sqrt(r_in(a) r_in(b)) and refactor          */
  VTM_Z_LEARNED = 3    /* learned impedances: opts.model maps the 8 features of each line end
                          (vtm_line_features) to log Z_e; both ends agree on
                          Z_t = exp((log Z_a + log Z_b) / 2) (Table 1 step 1)               */
};

enum vtm_precision {
  VTM_FP64 = 0,        /* factor, substitution and waves in FP64                              */
  VTM_FP32 = 1         /* factor, substitution and waves in FP32; FP64 residual and defect
                          correction around the sweeps (outer refinement)                     */
};

typedef struct vtm_mlp vtm_mlp;

typedef struct vtm_setup_opts {
  int32_t z_mode;          /* vtm_z_mode                                                     */
  double z_uniform;        /* UNIFORM: impedance (> 0)                                       */
  const double* z_lines;   /* EXPLICIT: host, nlines values (> 0)                            */
  int32_t precision;       /* vtm_precision                                                  */
  int32_t nrhs;            /* right-hand sides solved together: 1, 2, 4, 8, 16 or 32         */
  int32_t check_every;     /* sweeps between residual checks in vtm_solve (0 = 10)           */
  double inner_reduction;  /* FP32: restart the defect correction once the inner residual has
                              dropped by this factor (0 = 1e-4); ignored for FP64            */
  const vtm_mlp* model;    /* LEARNED: impedance model (not retained after vtm_setup)        */
  int64_t wait_polls;      /* polls of a bounded device wait before the sweep gives up and
                              reports VTM_ERR_TIMEOUT (0 = 4194304)                          */
  int32_t withhold_slab;   /* testing only: the sweep never issues the copy of this factor slab
                              of each subgraph, so that wait runs out (0 = off; k>0 = slab k-1) */
  int32_t sweep_variant;   /* 0 or 1: single-block sweep (the autotuner picks the staging depth);
                              2: pipelined sweep (nrhs <= 2; VTM_ERR_INVALID if no staging depth
                              fits).  The pipelined schedule is never chosen automatically: it
                              measured slower on every workload tried.
                              3: FP32, nrhs 16 / 32: the multi-RHS band sweep on the SIMT cores
                              only (by default its products run on the tensor cores when every
                              half-bandwidth is at most 384)                                   */
  int32_t sweep_form;      /* how a sweep obtains the port values u = P^T x_j (VTM_FORM_*):
                              BAND substitutes through the banded factor of K_j every sweep;
                              PORT precomputes the port response S_j = P^T K_j^{-1} P at setup
                              and updates the ports only (u = u_base + S_j s), running the band
                              substitution once per batch of sweeps to refresh the interior
                              unknowns; AUTO (0) takes PORT where it moves fewer bytes per sweep,
                              fits in shared memory (nrhs <= 8) and in device memory            */
  int32_t port_storage;    /* PORT form, FP32 solvers: storage of S_j (VTM_STORE_*).
                              nrhs <= 8: NATIVE (0) the solver precision; FP16 halves the bytes
                              of a sweep (each 32 x 32 tile of S_j scaled by its largest entry,
                              FP32 arithmetic; the sweeps then match the FP64 oracle to about
                              2^-11 per sweep and the FP64 defect correction restores the
                              tolerance; a phase on FP16 responses restarts once its inner
                              residual is below 4 x 2^-11, and with coupled lines once a check
                              gains less than a factor 2); FP16_AUTO takes FP16 when the
                              responses exceed 96 MB (streamed from HBM rather than held in L2),
                              and returns to FP32 for good once a defect-correction step gains
                              less than a factor 10.
                              nrhs 16 / 32 (tensor cores): S_j / sigma_j is kept as fp16 pairs
                              hi + lo (about 2^-22 relative); NATIVE and FP16_AUTO stream both
                              halves, FP16 streams the hi half only (half the bytes, 2^-11)    */
  /* Coupled lines (§7.2, Thm 7.1).  Lines that join the same two subgraphs form a bundle; a
   * conductance y_p >= 0 between two lines t, t' of one bundle makes the bundle's admittance
   * Y = Z^{-1} = diag(1/Z_t) + sum_p y_p (e_t - e_t')(e_t - e_t')^T, symmetric positive definite,
   * so Thm 7.1 applies.  Eq. 5.8 becomes K_j = Ã_j + P_j Y_j P_j^T and r_j = b̃_j + P_j Y_j w_in;
   * the wave update w_out = 2 u - w_in is unchanged.  The two copies that t and t' reach in each of
   * the two subgraphs must be neighbours there (an off-diagonal entry of Ã_j), so K_j keeps the
   * band of Ã_j; vtm_partition_line_pairs lists every such pair.  MATCHED impedances are computed
   * for the uncoupled lines and the couplings added afterwards.  VTM_ERR_INVALID: a line id out of
   * range, t == t', lines of different bundles, copies that are not neighbours, y < 0 or not
   * finite, or NULL arrays with ncouplings > 0. */
  int64_t ncouplings;          /* number of coupled pairs (0 = uncoupled lines)                  */
  const int64_t* couplings;    /* host, 2 x ncouplings line ids (t, t') per pair                 */
  const double* coupling_y;    /* host, ncouplings conductances y_p                              */
} vtm_setup_opts;

enum {
  VTM_STORE_NATIVE = 0,
  VTM_STORE_FP16 = 1,
  VTM_STORE_FP16_AUTO = 2
};

enum {
  VTM_FORM_AUTO = 0,
  VTM_FORM_BAND = 1,
  VTM_FORM_PORT = 2
};

typedef struct vtm_solver vtm_solver;

typedef struct vtm_solver_info {
  int32_t npieces;
  int64_t ncopies;
  int64_t nends;               /* 2 * nlines                                                  */
  int32_t nrhs;
  int32_t precision;
  int32_t block_rows;          /* substitution block height (rows per staged slab)            */
  int64_t factor_entries;      /* stored band entries (with padding)                          */
  int64_t band_entries;        /* structurally in-band entries sum_j (n_j (w_j+1) - w_j(w_j+1)/2) */
  int64_t factor_bytes;        /* stored factor bytes                                         */
  int64_t max_halfband;        /* max_j w_j                                                   */
  double setup_ms;             /* wall time of vtm_setup                                      */
  double factor_ms;            /* device time of the factorisation kernels                    */
  int32_t sweep_stages;        /* staged slabs per CTA chosen by the setup-time autotuner     */
  int32_t sweep_ctas_per_sm;   /* resident sweep CTAs per SM at that staging depth            */
  double sweep_ms;             /* autotuner's device time of one sweep (all subgraphs)        */
  int32_t flagged_pieces;      /* FP32 solvers: subgraphs refactored and swept in FP64 because
                                  their FP32 pivots broke down or kept < 1e-5 of the diagonal  */
  int32_t sweep_variant;       /* 0: one CTA works each block step in turn; 1: pipelined (warp 0
                                  finishes block k while the others prepare block k+1)        */
  int32_t sweep_form;          /* VTM_FORM_BAND or VTM_FORM_PORT (after AUTO was resolved)    */
  int64_t port_bytes;          /* PORT: bytes of the port responses S_j one sweep streams     */
  double port_setup_ms;        /* PORT: device time of computing S_j (unit-source solves)     */
  double port_sweep_ms;        /* PORT: device time of one port-form sweep                    */
  int64_t nports;              /* port copies (copies with at least one line end)             */
  int32_t port_storage_bits;   /* PORT: bits per stored S_j entry now (16, 32 or 64; FP16_AUTO
                                  turns 16 into 32 when it falls back)                         */
  int32_t factor_tc;           /* 1: the FP32 factorisation ran its trailing updates on the
                                  tensor cores (half-bandwidth 64 .. 384)                       */
  int64_t ncouplings;          /* coupled line pairs with y > 0 (0: uncoupled lines)           */
  int32_t band_tc;             /* 1: the multi-RHS band sweep (FP32, nrhs 16 / 32) runs its
                                  products on the tensor cores (factor balanced by its row norms,
                                  fp16 hi / lo panels of 128-row groups, FP32 accumulation)     */
  int64_t band_tc_bytes;       /* bytes of that tensor-core factor (each sweep reads it twice)  */
} vtm_solver_info;

/* Build the local matrices K_j = Ã_j + sum_e Z_e^{-1} e_c e_c^T (eq. 5.8), factor them on the
 * device once (banded Cholesky), allocate the wave and vector buffers.  `p` is not retained.
 * Errors: VTM_ERR_INVALID, VTM_ERR_NOT_SPD, VTM_ERR_OOM, VTM_ERR_CUDA. */
int vtm_setup(const vtm_partition* p, const vtm_setup_opts* opts, void* cuda_stream, vtm_solver** out);
int vtm_solver_get_info(const vtm_solver* s, vtm_solver_info* info);
/* Residual checks of the last vtm_solve, in order: sweeps done at the check, max_r relative
 * residual ||b_r - A x_r|| / ||b_r|| (FP64) and max_r inner residual (relative to the residual the
 * current defect-correction phase started from; equal to the former before the first restart).
 * Host arrays of *count entries; call with NULL arrays to read *count. */
int vtm_solver_get_history(const vtm_solver* s, int32_t* count, int32_t* sweeps, double* rel, double* inner);
void vtm_solver_destroy(vtm_solver* s);

/* ----------------------------------------------------------------------------------------------
 * Iteration (Table 1 steps 3-5)
 * --------------------------------------------------------------------------------------------*/

/* Split b into the subsystems' sources b̃_j (§4 step 3, eq. 4.4) for vtm_iterate.
 * b: host or device, column-major n x nrhs, leading dimension ldb.  Waves are not touched. */
int vtm_set_rhs(vtm_solver* s, const double* b, int64_t ldb);
/* Zero every wave (Table 1 step 2 with u^0 = omega^0 = 0). */
int vtm_reset(vtm_solver* s);
/* Run `sweeps` synchronous sweeps on the solver's stream (asynchronous): each sweep gathers the
 * incident wave of every line end from its twin (w_in[e] = w_out_prev[twin(e)]), solves every
 * K_j x_j = b̃_j + sum_e w_in[e]/Z_e e_c (eq. 5.8) with the stored factor (coupled lines:
 * b̃_j + P_j Y_j w_in, §7.2), and emits w_out[e] = 2 u_e - w_in[e] (the left side u - Z omega of
 * eq. 5.6 seen from the twin).
 * PORT form: the first sweeps - 1 sweeps update the ports only; the last one is a band sweep, so
 * the local solutions x_j (vtm_get_copies) always belong to the last sweep. */
int vtm_iterate(vtm_solver* s, int32_t sweeps);

/* Solve A x = b to max_r ||b_r - A x_r||_2 / ||b_r||_2 <= rtol (FP64 residual on the device,
 * checked every check_every sweeps), from zero waves.  FP32 solvers wrap the sweeps in FP64
 * defect correction.  b, x: host or device, column-major n x nrhs, leading dimension ld.
 * st may be NULL; vtm_solver_get_history returns the residual at every check.  Returns VTM_ERR_NOT_CONVERGED after maxit sweeps (x holds the last iterate),
 * VTM_ERR_DIVERGED on NaN/Inf. */
typedef struct vtm_stats {
  int32_t sweeps;          /* total sweeps                                        */
  int32_t checks;          /* residual evaluations                                */
  int32_t restarts;        /* defect-correction restarts                          */
  double rel_residual;     /* final max_r relative residual (FP64)                */
  double solve_ms;         /* wall time of the call                               */
  int32_t launches;        /* kernels of this library launched by the call        */
} vtm_stats;
int vtm_solve(vtm_solver* s, const double* b, double* x, int64_t ld, double rtol, int32_t maxit,
              vtm_stats* st);

/* Input impedance of every line end (Def. 7.1): with all sources zero, a unit inflow current at
 * the end's port and its own line open (every other line of the subgraph terminated by its
 * impedance), the port potential.  Computed on the device from the stored factors with unit
 * right-hand sides: g_c = (K_j^{-1})_{cc}, r_in(e) = g_c / (1 - g_c / Z_e).  Uncoupled lines
 * only (VTM_ERR_INVALID on a solver with couplings).
 * r_in: host, nends doubles in end order (2t = side a, 2t+1 = side b of line t).  Resets waves. */
int vtm_input_impedances(vtm_solver* s, double* r_in);
/* The line impedances the solver was set up with (after matching or the learned model), host,
 * nlines doubles in vtm_partition_get_lines order. */
int vtm_solver_get_impedances(const vtm_solver* s, double* z_lines);
/* Precision of each subgraph's factor and substitution: 32 or 64 (FP32 solvers refactor flagged
 * subgraphs in FP64), host int32 array of npieces. */
int vtm_solver_get_piece_precision(const vtm_solver* s, int32_t* bits);

/* Checkpoint / inspection.  Waves: outgoing waves of the last sweep, host, nends x nrhs
 * column-major (end order of vtm_partition_get_lines: end 2t = side a of line t, 2t+1 = side b).
 * Copies: the last local solutions, host, ncopies x nrhs column-major, copies numbered piece by
 * piece in local order.  vtm_get_copies needs a sweep to have run since vtm_reset. */
int vtm_get_state(vtm_solver* s, double* waves);
int vtm_set_state(vtm_solver* s, const double* waves);
int vtm_get_copies(vtm_solver* s, double* copies);

/* ----------------------------------------------------------------------------------------------
 * Learned impedance model (§7: the choice of Z is the preconditioner; §7.1 matching is the
 * paper's rule, the model is trained on impedances that the method finds by search)
 * --------------------------------------------------------------------------------------------*/

#define VTM_MLP_IN 8
#define VTM_MLP_HIDDEN 64
#define VTM_MLP_PARAMS 4801  /* W1[64][8], b1[64], W2[64][64], b2[64], W3[64], b3 (FP32 master) */

/* 8 features of every line end (its port copy c of vertex i in subgraph j), host float array of
 * nends x 8 (row e = end e in vtm_partition_get_lines order: 2t = side a, 2t+1 = side b):
 *   0 log a_ii            1 log a_ii^(c) (split weight of the copy, §4 step 3)
 *   2 log |O(i)| (copies)  3 lines at the copy (Fig. 7: 1, 2 or 3)
 *   4 log sum_{j in piece} |a_ij^(c)|   5 log a_ii^(twin copy)
 *   6 log(max_j |a_ij| / min_j |a_ij|) over the neighbours of i in A
 *   7 log(n / n_j) (how many subgraphs of this size the problem holds)                        */
int vtm_line_features(const vtm_partition* p, float* feats);

/* Model: 8 -> 64 -> 64 -> 1 perceptron, ReLU, BF16 weights with FP32 accumulation, output log Z.
 * Created with He-uniform weights from a SplitMix64 counter stream of `seed`; device memory owned
 * by the handle.  Parameters are exchanged as FP32 host arrays of VTM_MLP_PARAMS. */
int vtm_mlp_create(uint64_t seed, vtm_mlp** out);
void vtm_mlp_destroy(vtm_mlp* m);
int vtm_mlp_get_params(const vtm_mlp* m, float* params);
int vtm_mlp_set_params(vtm_mlp* m, const float* params);   /* also resets the Adam moments */
/* y[i] = model(X[i, :]); X: device n x 8 row-major float, y: device n floats. */
int vtm_mlp_forward(const vtm_mlp* m, const float* X, float* y, int64_t n, void* cuda_stream);
/* loss = mean_i (model(X_i) - target_i)^2 (returned on the host) and its gradient w.r.t. the BF16
 * weights, stored in the model (vtm_mlp_get_grads).  X, target: device. Synchronises the stream. */
int vtm_mlp_loss_grad(vtm_mlp* m, const float* X, const float* target, int64_t n, float* loss, void* cuda_stream);
int vtm_mlp_get_grads(const vtm_mlp* m, float* grads);
/* One Adam step on the FP32 master weights with the stored gradient; refreshes the BF16 copy. */
int vtm_mlp_adam_step(vtm_mlp* m, float lr, float beta1, float beta2, float eps, void* cuda_stream);

/* ----------------------------------------------------------------------------------------------
 * Allocation-free residual (the paper has no counterpart: this is a service for callers)
 * --------------------------------------------------------------------------------------------*/

/* Largest nrhs accepted by vtm_relative_residual_noalloc. */
#define VTM_NOALLOC_MAX_RHS 8

/* rel[r] = ||b_r - A x_r||_2 / ||b_r||_2 (||b_r - A x_r||_2 when b_r = 0) in FP64, for callers
 * that must not allocate device memory when they call it — e.g. a monitoring thread in a process
 * whose device memory is reserved up front by a framework's caching allocator, or a loop that
 * cannot afford cudaMalloc/cudaFree synchronising the device.  It calls no allocating routine:
 * its only scratch is a 128-byte file-scope device array (2 * VTM_NOALLOC_MAX_RHS doubles) that
 * every device holds, once it is loaded there (below), until the process exits.
 *   n, rowptr (n+1 int64), col (int32), val (double): A in full CSR, DEVICE memory.
 *   b, x: DEVICE, column-major n x nrhs with leading dimensions ldb, ldx >= n.
 *   rel: DEVICE, nrhs doubles (output).  nrhs in [1, VTM_NOALLOC_MAX_RHS], else VTM_ERR_INVALID.
 * Asynchronous on cuda_stream.  The first call on a device looks up the array's device address
 * (cudaGetSymbolAddress) with that device current; under CUDA's default lazy loading that look-up
 * also loads the array onto the device, which allocates device memory.  vtm_setup performs it for
 * its device; a caller that never calls vtm_setup makes one warm-up call per device before it
 * reserves device memory up front, and before any stream capture.  Later calls allocate nothing.
 * Every call reuses the same array (cleared at the start of each call), so calls that
 * overlap on the GPU — from two streams or two host threads — race and return wrong values:
 * serialise them. */
int vtm_relative_residual_noalloc(int64_t n, const int64_t* rowptr, const int32_t* col, const double* val,
                                  int32_t nrhs, const double* b, int64_t ldb, const double* x, int64_t ldx,
                                  double* rel, void* cuda_stream);

const char* vtm_last_error(void);
int vtm_version(void);

#ifdef __cplusplus
}
#endif
#endif /* VTM_H */
