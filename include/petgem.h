/* petgem.h - C ABI of the GB300 (sm_103a) hot path of the secondary-field CSEM forward solver.
 *
 * The method is the one of Castillo-Reyes, de la Puente and Cela, "PETGEM: A parallel code for
 * 3D CSEM forward modeling using edge finite elements" (Computers & Geosciences, 2018):
 *   curl curl E_s + i w mu0 sigma E_s = -i w mu0 (sigma - sigma_p) E_p        (Section 2, eq. 6)
 * with E_s = 0 on the outer boundary, discretised with lowest-order Nedelec edge elements on
 * tetrahedra (Section 3 eq. 9, Appendix B), the whole-space dipole primary field E_p
 * (Appendix A), a Krylov solve (Section 5.1 uses GMRES) and interpolation of E at receivers
 * (Section 3 eq. 7).  The calls follow the paper's problem statement (Section 4: physics,
 * mesh, solver and results sections of its parameters file).
 *
 * Conventions for every call:
 *   - Pointers documented as "device" are CUDA device pointers on the context's device; the
 *     caller owns them and keeps them alive until the call returns (for calls that only
 *     enqueue work: until the context stream has passed the work).  "host" pointers are read
 *     or written before the call returns.
 *   - Complex arrays are interleaved (re, im) pairs: complex128 = 2 doubles, complex64 = 2 floats.
 *   - All work is ordered on the stream given to petgem_create.  Calls that return a host
 *     scalar or struct synchronise that stream before returning.
 *   - Every call returns a status code (PETGEM_OK = 0).  No C++ exception crosses this ABI.
 *     petgem_last_error gives a message for the last failing call on a context.
 *   - A context is not thread-safe; use one context per host thread.
 */
#ifndef PETGEM_H
#define PETGEM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

/* ----------------------------------------------------------------------- status codes */
enum {
  PETGEM_OK = 0,
  PETGEM_ERR_INVALID_ARG = 1,     /* null pointer, bad size, call out of order */
  PETGEM_ERR_BAD_MESH = 2,        /* node id out of range, repeated node, non-manifold face */
  PETGEM_ERR_DEGENERATE_TET = 3,  /* a tet with zero volume */
  PETGEM_ERR_OUT_OF_MEMORY = 4,
  PETGEM_ERR_CUDA = 5,            /* a CUDA runtime error (message in petgem_last_error) */
  PETGEM_ERR_NOT_CONVERGED = 6,   /* iteration cap reached; info is still filled */
  PETGEM_ERR_BREAKDOWN = 7,       /* Krylov breakdown or a NaN/Inf in the iteration */
  PETGEM_ERR_RECEIVER_OUTSIDE = 8,/* a receiver lies in no tet; its outputs are NaN */
  PETGEM_ERR_UNSUPPORTED = 9,    /* a size or option the library does not handle */
  PETGEM_ERR_TIMEOUT = 10         /* a bounded device-side wait gave up; the call was abandoned */
};

/* ----------------------------------------------------------------------- types */
typedef struct petgem_ctx petgem_ctx; /* opaque; owns the library's device workspaces */

/* Electric dipole source of Appendix A (eqs. A.1-A.3): position (m), orientation and moment
 * I * dS (A m).  axis: 0 = x-, 1 = y-, 2 = z-directed. */
typedef struct {
  double x, y, z;
  double moment;
  int32_t axis;
  int32_t reserved;
} petgem_dipole;

enum { PETGEM_PREC_C128 = 0, PETGEM_PREC_MIXED = 1 };
enum { PETGEM_PRECOND_JACOBI = 0, PETGEM_PRECOND_LEARNED = 1, PETGEM_PRECOND_SSOR = 2 };

/* Solver options.  Restarted GMRES(restart), right-preconditioned by Jacobi D = diag(A),
 * x0 taken from the x argument, stopping when ||b - A x||_2 / ||b||_2 <= tol with the
 * residual recomputed in FP64 at every restart.
 *   precision = PETGEM_PREC_C128: every vector and the matrix in complex128.
 *   precision = PETGEM_PREC_MIXED: FP64 iterative refinement; each refinement step runs
 *     a GMRES cycle on a complex64 copy of the matrix with complex64 Krylov vectors (dot
 *     products summed in FP64 across the vector) until the inner residual falls by
 *     inner_tol or restart steps have run; x and the residual stay complex128.
 *   batch: number of sources iterated together (their SpMVs become one SpMM); 0 = all (groups
 *     of up to 32).  batch = 1 solves the sources one after the other.
 *   precond = PETGEM_PRECOND_LEARNED: flexible GMRES whose every step uses the learned
 *     auxiliary-space preconditioner z = M^{-1} v (petgem_learned_create; in the Jacobi-scaled
 *     variables D M^{-1} v) from the first cycle on.  Sources one by one (batch = 1): classical
 *     Gram-Schmidt with a second pass when the norm fell below 1/sqrt(10).  Sources together
 *     (batch != 1): the block solve above, with the network applied to every live source's
 *     column in each step and one SpMM on the block of preconditioned vectors; classical
 *     Gram-Schmidt, one pass.  A learned cycle that removes less than 10 % of a source's FP64
 *     residual is undone and that source continues with Jacobi alone (info.fell_back).
 *   precond = PETGEM_PRECOND_SSOR (method SQMR only; PETGEM_ERR_UNSUPPORTED otherwise):
 *     symmetric SOR, the preconditioner of the paper's Section 5.3 runs, in the order of a
 *     multicolour colouring of the matrix graph (petgem_colouring): with A = D + L + U split by
 *     colour, M = (D + omega L) D^{-1} (D + omega U), applied to SQMR as the symmetric split
 *     M1 = (D + omega L) D^{-1/2}, M2 = M1^T.  Each SQMR step costs a forward and a backward
 *     sweep (one launch per colour each) besides the product.  Precision as for COCG: FP64
 *     residuals around inner solves in complex64 (MIXED) or complex128 (C128).  Sources are
 *     solved one after the other (`batch` and `use_graphs` are ignored); `omega` sets the
 *     relaxation factor. */
typedef struct {
  int32_t restart;
  int32_t precision;
  int32_t precond;
  int32_t batch;
  double tol;
  double inner_tol;
  int64_t max_iters;   /* cap on Krylov iterations per source */
  int32_t orth;        /* Arnoldi orthogonalisation: PETGEM_ORTH_CGS (default), _CGS2, _CGS_IFNEEDED */
  int32_t use_graphs;  /* 1 = replay each GMRES restart cycle as a CUDA graph, captured once per
                          solve configuration (Jacobi or learned preconditioner; ignored while
                          kernel profiling is on, and by COCG, whose iterations run in one
                          persistent kernel); results are identical to direct launches */
  int32_t method;      /* PETGEM_METHOD_GMRES (default), PETGEM_METHOD_COCG or PETGEM_METHOD_SQMR */
  int32_t spmv_lanes;  /* petgem_solve_batch: layout of the sparse product: 2, 4 or 8 = CSR with that
                          many lanes per row, 1 = SELL-32 with rows grouped by edge kind (CSR with
                          4 lanes when a mesh lacks that layout); 0 = chosen by the autotuner.
                          petgem_solve with several sources iterated together (batch != 1): the
                          block SpMM, 0 = chosen by the autotuner (once per context and problem
                          shape: rows, nonzeros, sources, precision), 1 = one lane per (row, source),
                          16 / 32 / 64 = the staged kernel with that band height (other values:
                          PETGEM_ERR_UNSUPPORTED); ignored by single-source solves (which use
                          SELL-32 when the mesh has it) */
  double omega;        /* SSOR relaxation factor, 0 < omega < 2; 0 = 1 (symmetric Gauss-Seidel) */
} petgem_solve_opts;

/* Krylov method.
 *   GMRES: restarted GMRES(restart) as above.
 *   COCG: conjugate orthogonal conjugate gradient for the complex-symmetric matrix (A^T = A),
 *     the short-recurrence family the paper's Section 5.3 solves with (symmetric QMR): CG with
 *     the bilinear form u^T v, Jacobi as the symmetric scaling D^{-1/2} A D^{-1/2}, no basis
 *     stored.  precision MIXED: complex64 inner solves that each reduce the scaled residual by
 *     inner_tol, restarted from the FP64 residual b - A x; C128: FP64 throughout.  `restart` is
 *     the number of iterations between host checks of the device-side stopping flag; `batch`
 *     groups sources as for GMRES (their SpMVs become one SpMM; each source keeps its own scalars,
 *     normalisation and stopping test); `orth` is ignored; precond must be Jacobi
 *     (PETGEM_ERR_UNSUPPORTED otherwise).
 *     info.restarts counts the inner solves.  A breakdown of the bilinear form (p^T A p = 0) ends
 *     an inner solve early; one at the very first step returns PETGEM_ERR_BREAKDOWN. */
/*   SQMR: symmetric QMR, the solver of the paper's Section 5.3: the Lanczos recurrences of COCG
 *     (same residuals, directions and scalars) with the quasi-minimal-residual iterate, which
 *     smooths COCG's residual history; each inner solve stops when the quasi-residual norm tau
 *     fell by inner_tol.  Jacobi as for COCG (the symmetric split D^{1/2} D^{1/2}); sources are
 *     solved one after the other (`batch` is ignored); otherwise as COCG. */
enum { PETGEM_METHOD_GMRES = 0, PETGEM_METHOD_COCG = 1, PETGEM_METHOD_SQMR = 2 };

/* Orthogonalisation of each new Krylov vector w against the basis V:
 *   CGS: classical Gram-Schmidt once (two passes over V per step; the default of PETSc's GMRES);
 *   CGS2: classical Gram-Schmidt twice (three passes);
 *   CGS_IFNEEDED: a second pass only when ||w|| fell below 1/sqrt(10) of its value (one classical
 *     pass loses orthogonality in proportion to that cancellation). */
enum { PETGEM_ORTH_CGS2 = 0, PETGEM_ORTH_CGS = 1, PETGEM_ORTH_CGS_IFNEEDED = 2 };

/* Per-source results of petgem_solve. */
typedef struct {
  int64_t iters;       /* Krylov iterations (SpMVs inside Arnoldi) */
  int64_t restarts;    /* GMRES cycles */
  int64_t refinements; /* FP64 residual evaluations after the first */
  double true_rel_residual; /* ||b - A x|| / ||b|| in FP64 at exit */
  int32_t status;      /* PETGEM_OK, PETGEM_ERR_NOT_CONVERGED, _BREAKDOWN or _TIMEOUT */
  int32_t reorth;      /* Arnoldi steps that needed a second Gram-Schmidt pass */
  int32_t fell_back;   /* learned preconditioner: 1 if the solve switched back to Jacobi */
  int32_t spmv_lanes;  /* petgem_solve_batch: the product's layout it ran with (as in the options:
                          1 = SELL-32, 2 / 4 / 8 = CSR lanes per row).  Multi-source block solves
                          (batch != 1): the block SpMM the autotuner chose for this mesh and group
                          size, 16 / 32 / 64 = the band height of the staged kernel (each band's
                          distinct rows of the block vector copied to shared memory once), 1 = one
                          lane per (row, source) reading the block vector directly.  0 otherwise */
} petgem_solve_info;

/* ----------------------------------------------------------------------- lifecycle */
/* Create a context bound to CUDA device `device`, ordering all work on `cuda_stream`
 * (a cudaStream_t; NULL = the legacy default stream). */
int petgem_create(petgem_ctx **out, int device, void *cuda_stream);
/* Free every device buffer the context owns.  NULL is accepted. */
int petgem_destroy(petgem_ctx *ctx);
const char *petgem_status_string(int status);
const char *petgem_last_error(const petgem_ctx *ctx);

/* ----------------------------------------------------------------------- mesh (Appendix B) */
/* Global edge numbering and orientation, boundary edges and the sparse pattern.
 * nodes: device double[n_nodes][3] (m).  tets: device int32[n_tets][4] node ids (0-based),
 *   either orientation.
 * Local edge i of a tet joins local nodes (a, b) = (1,2), (1,3), (1,4), (2,3), (4,2), (3,4)
 * (Appendix B eqs. B.1-B.6, 1-based).  A global edge runs from its lower to its higher node
 * id and its sign in a tet is +1 when the local edge runs the same way (eq. B.16).  Global
 * edge ids are the ranks of (low id, high id) in lexicographic order, so the numbering is
 * unique.  Boundary edges are the edges of faces held by exactly one tet (Dirichlet edges of
 * Section 2).  The sparse pattern has one row per edge: interior rows hold the interior
 * columns they couple to, boundary rows hold their diagonal only.
 * n_edges_out: host; receives the edge count (synchronises the stream).
 * Errors: PETGEM_ERR_BAD_MESH (ids out of range, repeated node, face in more than two tets),
 * PETGEM_ERR_UNSUPPORTED (n_tets >= 2^31 / 36 or n_nodes >= 2^31). */
int petgem_mesh_edges(petgem_ctx *ctx, int64_t n_nodes, const double *nodes, int64_t n_tets,
                      const int32_t *tets, int64_t *n_edges_out);

/* Copy the topology out (each pointer optional, device): edges int32[E][2] (low, high),
 * tet_edges int32[T][6], signs int8[T][6] in {+1, -1}, boundary uint8[E] in {0, 1}. */
int petgem_get_topology(petgem_ctx *ctx, int32_t *edges, int32_t *tet_edges, int8_t *signs,
                        uint8_t *boundary);

/* ----------------------------------------------------------------------- assembly (Section 3) */
/* Element matrices and right-hand sides, global assembly and Dirichlet rows (eqs. 6 and 9):
 *   A = sum_e K^e + i w mu0 sigma_e M^e,  b_s = sum_e -i w mu0 (sigma_e - sigma_p) R^e_s,
 *   R^e_{s,k} = int_e S_k N_k . E_p(x; source s, sigma_p) dV,
 * w = 2 pi freq_hz, mu0 = 4 pi 1e-7 H/m.  K^e and M^e are the closed forms of eqs. B.14-B.15;
 * R^e uses the symmetric 4-point degree-2 rule and is skipped where sigma_e = sigma_p.
 * Boundary rows become identity rows with b = 0.  Contributions are summed in a fixed order,
 * so repeated calls give bit-identical results.
 * sigma: device double[n_tets] (S/m, > 0).  src: host petgem_dipole[n_src].
 * Requires petgem_mesh_edges.  Errors: PETGEM_ERR_DEGENERATE_TET, PETGEM_ERR_INVALID_ARG. */
int petgem_assemble(petgem_ctx *ctx, double freq_hz, const double *sigma, double sigma_p,
                    int32_t n_src, const petgem_dipole *src);

/* Another frequency (and set of sources) on the same mesh, conductivities and background sigma_p
 * as the last petgem_assemble: eq. 9 is linear in w, A(w) = K + i w mu0 M_sigma with the real
 * global matrices K = sum_e K^e and M_sigma = sum_e sigma_e M^e, which petgem_assemble keeps; this
 * call forms A and diag(A) from them (one pass over the matrix entries instead of the element
 * matrices and their gather) and computes the right-hand sides for the new frequency and
 * sources.  petgem_assemble itself forms A the same way, so the two give bit-identical systems.
 * src: host petgem_dipole[n_src].  Errors: PETGEM_ERR_INVALID_ARG (no petgem_assemble before,
 * freq_hz <= 0, n_src < 1, a bad dipole). */
int petgem_assemble_frequency(petgem_ctx *ctx, double freq_hz, int32_t n_src, const petgem_dipole *src);

/* Copy the assembled system out.  nnz_out: host (synchronises).  row_ptr int64[E+1],
 * col int32[nnz], val complex128[nnz], b complex128[n_src][E], diag complex128[E] (each device,
 * optional).  Rows list columns in increasing order. */
int petgem_get_system(petgem_ctx *ctx, int64_t *nnz_out, int64_t *row_ptr, int32_t *col, void *val,
                      void *b, void *diag);

/* Element matrices as computed by the assembly kernel: K, M device double[21][n_tets], the
 * upper triangle (i <= j, row-major order of (i, j)) of the signed 6x6 matrices; vol device
 * double[n_tets] (optional). */
int petgem_get_elements(petgem_ctx *ctx, double *K21, double *M21, double *vol);

/* ----------------------------------------------------------------------- solve (Section 5.1) */
/* Solve A x_s = b_s for every source.  x: device complex128[n_src][E]; the initial guess in,
 * the solution out.  info: host petgem_solve_info[n_src].  opts: host (NULL = defaults:
 * restart 50, c128, Jacobi, tol 1e-8, max_iters 200000, inner_tol 1e-4, orth CGS).
 * Returns PETGEM_ERR_NOT_CONVERGED or PETGEM_ERR_BREAKDOWN if any source ended that way. */
int petgem_solve(petgem_ctx *ctx, const petgem_solve_opts *opts, void *x, petgem_solve_info *info);

/* Solve the systems of several contexts together: one mesh per context (sizes may differ), every
 * (context, source) pair one system A_k x = b_ks, with COCG (opts->method must be
 * PETGEM_METHOD_COCG, precond Jacobi; precision MIXED or C128 as for petgem_solve).
 * The inner iterations of all systems run in one persistent cooperative launch per refinement
 * round (the blocks of the GPU divided among the systems by a scheduler in proportion to each
 * system's matrix entries times its expected iterations, re-divided every round from the
 * iterations each system took); the FP64 refinement steps of all systems (solution update, true
 * residual, its norm, the stopping decision, the next start) run as one launch sequence per
 * round, replayed as a CUDA graph when opts->use_graphs = 1.  opts->spmv_lanes = 0 lets an
 * autotuner pick the sparse product's layout (CSR with 2, 4 or 8 lanes per row, or SELL-32 when
 * every mesh has it) by timing a few iterations with each before the first inner solve.
 * The contexts must share a device and each must have called petgem_assemble.  The work runs on
 * ctxs[0]'s stream, after the work already queued on every context's stream and before any work
 * queued on them afterwards.
 *   ctxs: host array of n_ctx contexts (n_ctx = 0: nothing to do).
 *   x: host array of n_ctx device pointers, x[k] complex128[n_src_k][E_k] (x0 in, solution out).
 *   info: host array of sum_k n_src_k entries, context by context, source by source.
 *   The workspace belongs to ctxs[0] (freed by its petgem_destroy).
 * Errors: PETGEM_ERR_INVALID_ARG (null arguments, a context not assembled, contexts on different
 * devices), PETGEM_ERR_UNSUPPORTED (method GMRES, the learned preconditioner, more than 64
 * systems, spmv_lanes not in {0, 2, 4, 8}), PETGEM_ERR_NOT_CONVERGED / _BREAKDOWN / _TIMEOUT when a
 * system ended so (info is still filled); the error text is ctxs[0]'s. */
int petgem_solve_batch(petgem_ctx *const *ctxs, int32_t n_ctx, const petgem_solve_opts *opts, void *const *x,
                       petgem_solve_info *info);

/* y = A x for the assembled matrix (complex128, device, n_src = 1 vector of E entries). */
int petgem_spmv(petgem_ctx *ctx, const void *x, void *y);

/* Multicolour ordering of the SSOR preconditioner (Jones and Plassmann's parallel colouring):
 * row i has the priority key (splitmix64(i), i), splitmix64 being the output function of Steele,
 * Lea and Flood's SplitMix64 generator for the state i (add 0x9E3779B97F4A7C15; xor-shift 30,
 * multiply by 0xBF58476D1CE4E5B9; xor-shift 27, multiply by 0x94D049BB133111EB; xor-shift 31;
 * all modulo 2^64), keys compared lexicographically.  Each round, every uncoloured row whose key
 * exceeds those of all its uncoloured neighbours (the off-diagonal columns of its pattern row)
 * takes the smallest colour none of its coloured neighbours holds: the greedy colouring in
 * decreasing key order.  Needs petgem_mesh_edges; computed once per mesh.
 *   colour: device int32[E] (optional) receives each row's colour.
 *   n_colours, n_rounds: host (optional) receive the number of colours and of rounds.
 * Synchronises the stream.  Errors: PETGEM_ERR_UNSUPPORTED when a row would need more than 64
 * colours (a row with more than 63 neighbours) or E >= 2^31. */
int petgem_colouring(petgem_ctx *ctx, int32_t *colour, int32_t *n_colours, int32_t *n_rounds);

/* z = M^{-1} r for the SSOR preconditioner above (forward sweep, scaling by D, backward sweep),
 * in FP64.  r, z: device complex128[E] in the edge order, caller-owned, distinct (r is only read).
 * omega as in petgem_solve_opts (0 = 1).  Needs petgem_assemble; computes the colouring first if
 * the mesh has none yet.  Synchronises the stream.
 * Errors: PETGEM_ERR_INVALID_ARG (not assembled, null or aliased vectors, omega outside (0, 2)),
 * the colouring's errors (petgem_colouring). */
int petgem_ssor_apply(petgem_ctx *ctx, double omega, const void *r, void *z);

/* ----------------------------------------------------------------------- receivers (eq. 7) */
/* Field at receiver points.  rx: device double[n_rcv][3].  x: device complex128[n_src][E]
 * (edge DOFs, e.g. from petgem_solve).  out: device complex128[n_src][n_rcv][3][3], the
 * innermost pair of axes being (kind, component) with kind 0 = E_p (sigma_p), 1 = E_s =
 * sum_i S_i N_i(x) x_g(i) (eq. 7), 2 = E_p + E_s.  A receiver belongs to the lowest-id tet
 * whose barycentric coordinates are all >= -1e-12.  Returns PETGEM_ERR_RECEIVER_OUTSIDE when
 * some receiver is in no tet (its nine outputs are NaN). */
int petgem_receivers(petgem_ctx *ctx, int32_t n_rcv, const double *rx, const void *x, void *out);

/* ----------------------------------------------------------------------- layered background */
/* Primary field of a horizontal electric dipole in a horizontally layered Earth (Section 2: for a
 * layered background the primary field is computed semi-analytically by Hankel transforms, where
 * the paper uses filters it does not give).  The field is App. A's whole-space field of the source
 * layer's conductivity plus Hankel integrals of the difference between the layered and the
 * whole-space TE/TM mode spectra, evaluated by a fixed 8-point Gauss-Legendre panel rule:
 * lambda_max = 36 / D (D = the shortest source - interface - point path for a point in the source
 * layer, else |z - z_s|, at least 1e-3 m), the panel [0, k_min / 16] (k_min = min_j sqrt(w mu0
 * sigma_j)), panels doubling up to w = min(pi / rho, lambda_max / 16), then width w, at most 16384.
 * Same conventions as App. A (operator curl curl + i w mu0 sigma, e^{-ikr} decay).
 *   n_layers: 1..8, top first.  z_interfaces: host double[n_layers - 1], strictly decreasing (z up);
 *   layer 0 lies above z_interfaces[0]; a point on an interface belongs to the layer above.
 *   sigma_layers: host double[n_layers] (S/m, > 0).  src: host, axis 0 or 1 (horizontal dipoles).
 *   pts: device double[n_pts][3]; out: device complex128[n_pts][3] (E_x, E_y, E_z), overwritten.
 * Work is enqueued on `stream` (the call returns at once; nothing is allocated).
 * Errors (nothing launched): null pointers, n_pts < 0, freq <= 0, interfaces not decreasing or a
 * conductivity <= 0: PETGEM_ERR_INVALID_ARG; more than 8 layers or a vertical dipole:
 * PETGEM_ERR_UNSUPPORTED. */
int petgem_primary_layered(void *stream, int32_t n_layers, const double *z_interfaces, const double *sigma_layers,
                           double freq_hz, const petgem_dipole *src, int32_t n_pts, const double *pts, void *out);

/* Assembly with a layered background (Section 2, eq. 6 with sigma_p(z) layered): as
 * petgem_assemble, with the primary field of petgem_primary_layered and delta sigma_e = sigma_e -
 * (conductivity of the layer holding the tet's centroid), so only tets that differ from their
 * layer carry a right-hand side.  The background stays with the context: petgem_assemble_frequency
 * re-forms the right-hand sides in it, and petgem_receivers reports E_p of the layered background
 * (kind 0) and E_p + E_s.  The context's sigma_p (network features) becomes the conductivity of the
 * first source's layer.  petgem_assemble returns the context to a homogeneous background.
 * z_interfaces, sigma_layers: host, as for petgem_primary_layered; sigma: device double[n_tets];
 * src: host, horizontal dipoles.  Errors as petgem_assemble, plus PETGEM_ERR_UNSUPPORTED for more
 * than 8 layers or a vertical dipole. */
int petgem_assemble_layered(petgem_ctx *ctx, double freq_hz, const double *sigma, int32_t n_layers,
                            const double *z_interfaces, const double *sigma_layers, int32_t n_src,
                            const petgem_dipole *src);

/* ----------------------------------------------------------------------- learned preconditioner */
/* Not in the paper (it solves with GMRES, SQMR and MUMPS, Sections 5.1-5.3).  An additive
 * auxiliary-space preconditioner for the edge-element system (Hiptmair-Xu decomposition) whose
 * two nodal solves are replaced by a 3-D convolutional network on the node grid of a Kuhn-split
 * lattice of nx x ny x nz cells (node ids i + (nx+1) (j + (ny+1) k), every edge a step +x, +y,
 * +z, +xy, +xz, +yz or +xyz from its low node):
 *     z = M^{-1} r = D^{-1} r + G phi + Pi w,
 * with D = diag(A), (G phi)_e = (phi_hi - phi_lo) / |t_e| (nodal gradients, which the curl-curl
 * term annihilates), (Pi w)_e = (w_lo + w_hi) . t_e / (2 |t_e|) (nodal vector fields), t_e =
 * x_hi - x_lo, and phi, w zero on the outer boundary.  Network input (16 channels per node): with
 * sg = |diag(G^T A G)|^{-1/2}, sp = |diag(Pi^T A Pi)|^{-1/2} (per axis; zero on boundary nodes),
 * fg = sg G^T r, fp = sp Pi^T r, s = the RMS of (fg, fp) over the interior nodes' four complex
 * values: Re fg / s, Im fg / s, Re fp / s (x, y, z), Im fp / s (x, y, z), log10(sigma / sigma_p),
 * log10(w mu0 sigma h^2) of the cell whose lowest corner is the node (h = the first cell's
 * geometric-mean spacing), and six zeros.  Output channels: phi = s sg (y0 + i y1), w = s sp
 * (y2..4 + i y5..7); channels 8..15 unused.  Four levels (the node grid and three 2x poolings),
 * seven 3x3x3 convolutions (16/32 channels, BF16 operands on the tensor cores, FP32 accumulation
 * and FP32 master weights), ReLU, skip additions.
 * petgem_learned_create: after petgem_mesh_edges on such a lattice; keeps the parameters when
 *   called again for another mesh (the network is fully convolutional).  PETGEM_ERR_UNSUPPORTED
 *   if some edge is not a lattice step.
 * petgem_learned_params: host float[n] in (set) / out (get, and grad = the gradient accumulated by
 *   the last train step, scaled by 1 / n_samples); NULL to skip; *n_params receives the count.
 * petgem_learned_train_step: one Adam step (lr) on the mean over n_samples solver iterates
 *   x_iters (device complex128 [n_samples][E], e.g. the iterate at the start of every GMRES cycle)
 *   of the residual angle L = 1 - |<r, A z>|^2 / (|r|^2 |A z|^2), r = b - A x of the assembled
 *   system (source 0), z = M^{-1} r: zero when one step along z removes the whole residual.
 *   *loss (host) receives the mean L.
 * petgem_learned_apply: z = M^{-1} r for one device complex128 vector r of E entries. */
int petgem_learned_create(petgem_ctx *ctx, int32_t nx, int32_t ny, int32_t nz);
int petgem_learned_params(petgem_ctx *ctx, const float *set, float *get, float *grad, int64_t *n_params);
int petgem_learned_train_step(petgem_ctx *ctx, int32_t n_samples, const void *x_iters, float lr, double *loss);
int petgem_learned_apply(petgem_ctx *ctx, const void *r, void *z);

/* The network's tensor-core kernels as plain functions (test and diagnostic entry points):
 * grids are gx x gy x gz voxels (v = x + gx (y + gy z)), activations BF16 [V][C], weights BF16
 * [27][cout][cin] with tap t = (dx+1) + 3 (dy+1) + 9 (dz+1), zero "same" padding; cin, cout in
 * {16, 32}.  petgem_nn_conv3d: y[v][co] = bias[co] + sum_t,ci W[t][co][ci] x[v + d_t][ci], ReLU
 * when relu != 0, y BF16 (y_fp32 = 0) or FP32 [V][cout].  petgem_nn_conv3d_wgrad: dw[t][co][ci] =
 * sum_v dy[v][co] x[v + d_t][ci] (FP32).  All pointers device; work ordered on `stream`.
 * petgem_nn_conv3d's x, w and y must be 16-byte aligned (the kernel copies 8 channels, 16 bytes,
 * at a time into shared memory and stores its output in 16-byte pieces).
 * Errors: a dimension < 1, a null pointer, or (petgem_nn_conv3d) an x, w or y not 16-byte
 * aligned: PETGEM_ERR_INVALID_ARG; gx gy gz 32 >= 2^31 (the kernels index voxel channels in 32
 * bits) or cin / cout not in {16, 32}: PETGEM_ERR_UNSUPPORTED, nothing launched. */
int petgem_nn_conv3d(void *stream, int32_t gx, int32_t gy, int32_t gz, int32_t cin, int32_t cout, const void *x,
                     const void *w, const float *bias, int32_t relu, void *y, int32_t y_fp32);
int petgem_nn_conv3d_wgrad(void *stream, int32_t gx, int32_t gy, int32_t gz, int32_t cin, int32_t cout, const void *x,
                           const void *dy, float *dw);

/* Allocation-free form of petgem_nn_conv3d_wgrad.  The paper has no counterpart: it is an
 * integration entry point.  Same arguments, layouts and result (dw FP32 [27][cout][cin], device,
 * overwritten; x, dy device, read only; work ordered on `stream`, which must belong to the
 * current device; returns after the stream has passed the work).  For callers that cannot
 * allocate device memory during the call (a framework whose caching allocator holds the free
 * memory, or a step run with allocation forbidden because an allocation can wait on a lock and
 * a release can synchronise the device): it calls no cudaMalloc, cudaMallocAsync, cudaFree or
 * other allocating routine, and works in a fixed scratch array of the library's device code
 * (3.4 MB per device) that holds grids of at most PETGEM_NOALLOC_MAX_VOXELS voxels.
 *   - any of gx, gy, gz or their product > PETGEM_NOALLOC_MAX_VOXELS (each dimension is checked
 *     before the product is formed, so no product wraps), or cin / cout not in {16, 32}: PETGEM_ERR_UNSUPPORTED,
 *     nothing launched and dw untouched.  Null pointer or a dimension < 1: PETGEM_ERR_INVALID_ARG.
 *   - The first call on a device looks the scratch's address up (cudaGetSymbolAddress, with that
 *     device current; PETGEM_ERR_CUDA if it fails); make that first call before any stream capture.
 *   - All calls on a device share the scratch: calls that overlap in time (two streams, two host
 *     threads) race on it and give wrong results.  Serialise them. */
#define PETGEM_NOALLOC_MAX_VOXELS 131072
int petgem_nn_conv3d_wgrad_noalloc(void *stream, int32_t gx, int32_t gy, int32_t gz, int32_t cin, int32_t cout,
                                   const void *x, const void *dy, float *dw);

/* ----------------------------------------------------------------------- measurement */
/* Per-kernel device time recorded with CUDA events around launches while enabled.
 * petgem_profile(ctx, 1) clears and enables, 0 disables.  petgem_kernel_stats returns, for
 * kernel `name` (e.g. "spmv_c64"), the launch count, total milliseconds and the algorithmic
 * bytes those launches moved (synchronises).  For the network's tensor-core convolutions
 * ("conv3d_fwd") the third value counts floating-point operations (2 per multiply-add). */
int petgem_profile(petgem_ctx *ctx, int enable);
int petgem_kernel_stats(petgem_ctx *ctx, const char *name, int64_t *launches, double *total_ms,
                        double *bytes);
/* Number of kernel launches the context has issued since creation (host counter). */
int64_t petgem_launch_count(const petgem_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* PETGEM_H */
