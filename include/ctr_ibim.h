/*
 * ctr_ibim.h -- C ABI of the GB300 CTR-IBIM engine.
 *
 * Solves the linearized Poisson-Boltzmann interface problem (Eq. 1.1) through
 * the boundary integral pair of Eqs. (1.2)-(1.3), written as volume integrals
 * over a tube around the surface (Sec. 2.1, Eq. 2.13) and discretized on the
 * grid nodes of the tube by the corrected trapezoidal rule (Sec. 2.2,
 * Eqs. 2.14-2.15; matrix form Eq. 2.30, corrections of Sec. 2.4).
 *
 * Conventions shared by every entry point:
 *   - Units are those of the paper (lengths in Angstrom, charges in e,
 *     G0 = 1/(4 pi r), no Coulomb constant).
 *   - Grid node (i, j, k) sits at origin + h (i, j, k); grid arrays are flat,
 *     x fastest: index i + nx (j + ny k).
 *   - The signed distance is positive OUTSIDE the molecule (the paper, Sec.
 *     2.1, uses the opposite sign); the normal grad d then points outward.
 *   - The M unknown nodes are the grid nodes with |d| < eps, in increasing
 *     grid index; vectors of unknowns are p = [rho1 (M); rho2 (M)], rho1 the
 *     potential psi, rho2 its interior normal derivative (Eq. 2.13).
 *   - "Host" pointers are ordinary CPU memory; with on_device != 0 the
 *     pointer must be CUDA device memory of the handle's device.  The caller
 *     owns every buffer it passes; the library copies inputs and keeps no
 *     caller pointer after a call returns.
 *   - Every call returns CTR_OK (0) on success, CTR_NOT_CONVERGED (1) when a
 *     solve stops at its iteration limit (outputs are still written), or a
 *     negative status.  ctr_last_error() gives a message for the calling
 *     thread.  No C++ exception crosses this interface.
 *   - One handle is used by one host thread at a time.  All device work of
 *     a handle runs on the stream given at setup; calls return after that
 *     stream has finished the call's work (results are ready).
 */
#ifndef CTR_IBIM_H
#define CTR_IBIM_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define CTR_OK 0
#define CTR_NOT_CONVERGED 1
#define CTR_ERR_INVALID (-1)       /* a bad argument (null pointer, size, option) */
#define CTR_ERR_EMPTY_TUBE (-2)    /* no grid node with |d| < eps */
#define CTR_ERR_GRID_MARGIN (-3)   /* a tube node lies within 2 nodes of the grid boundary */
#define CTR_ERR_CUDA (-4)          /* a CUDA runtime error */
#define CTR_ERR_NOMEM (-5)         /* device allocation failed */
#define CTR_ERR_NUMERIC (-6)       /* a non-finite value appeared (geometry or solve) */
#define CTR_ERR_DEVICE_WAIT (-7)   /* a kernel gave up a bounded wait (internal error) */
#define CTR_ERR_CAPACITY (-8)      /* request larger than a fixed capacity */
#define CTR_ERR_CANCELLED (-9)     /* a server request was cancelled before it finished */

/*
 * Arithmetic of the dense pair sums (the correction, the diagonal, vectors
 * and the Krylov algebra are FP64 in every mode):
 *   CTR_FP64         IEEE FP64 (DFMA).
 *   CTR_FP32_REFINE  FP32 pair terms, per-tile FP32 sums added in FP64; as a
 *                    solve mode, GMRES on this operator inside FP64-accurate
 *                    iterative refinement.
 *   CTR_DF64         double-FP32 ("float-float") arithmetic on the FP32 pipe:
 *                    every quantity a pair of floats, about 2^-44 relative
 *                    accuracy, within 1e-12 of the FP64 operator.
 */
enum { CTR_FP64 = 0, CTR_FP32_REFINE = 1, CTR_DF64 = 2 };

/*
 * Quadrature of the rows (Secs. 2.3, 2.4, 3.2):
 *   CTR_METHOD_HYB   HYB-IBIM: CTR2 corrections (Sec. 2.4) at "good" nodes;
 *                    K-reg rows and J = 1 (Eq. 3.2) at "bad" nodes, a node being
 *                    bad when a finite-difference curvature is non-finite or
 *                    |k_i| (eps + h) >= 0.8 (the tube would reach within 20% of
 *                    the focal distance).  On smooth surfaces resolved by the
 *                    grid no node is bad and this is plain CTR2.
 *   CTR_METHOD_KREG  K-reg everywhere (Sec. 2.3), J = 1 everywhere.
 */
enum { CTR_METHOD_HYB = 0, CTR_METHOD_KREG = 1 };

/*
 * Evaluation of the dense sum of Eq. (2.30) (Sec. 2.5 accelerates it with a
 * black-box fast multipole method and gives no parameters):
 *   CTR_FARFIELD_DIRECT    every pair, M^2 per operator application.
 *   CTR_FARFIELD_TREECODE  a particle-cluster treecode.  An octree over the
 *       tube nodes' integer grid indices (leaves of at most tree_leaf nodes)
 *       orders the nodes; for each target block, a cluster that is well
 *       separated from it (theta |c_B - c_C| > r_B + r_C on the integer boxes
 *       widened by ceil(eps/h) grid units, decided exactly), that holds none of
 *       the block's correction nodes and that has more than (degree+1)^3 nodes
 *       (half of that for the float-float arithmetic, whose direct pairs cost
 *       about two of its float-float proxy evaluations each)
 *       is replaced by (degree+1)^3 tensor Chebyshev points on the tight box of
 *       its points P carrying interpolated charges (barycentric Lagrange
 *       interpolation of the kernels' source variable, d/dn_y on the basis);
 *       every other pair is summed directly with the correction pairs skipped
 *       exactly.  The error against the direct sum falls geometrically with the
 *       degree (about 6e-8 relative at degree 10, theta 0.8; the CTR_FP32_REFINE
 *       operator, which only drives the inner GMRES, uses its own degree and
 *       theta, 6 and 0.9 by default: about 7e-6).  The far field has the
 *       arithmetic of its operator: FP32 charges and evaluations for
 *       CTR_FP32_REFINE, FP64 charges and float-float evaluations for CTR_DF64,
 *       FP64 for CTR_FP64; the direct part keeps the arithmetic's pair kernels.
 *       The CTR_DF64 and CTR_FP64 treecode operators are consistent to their
 *       arithmetic's rounding, so refinement reaches tolerances like 1e-10 (the
 *       solution is then that of the treecode operator, within the
 *       interpolation error of the direct sum's).  A CTR_FP32_REFINE treecode
 *       solve forms every refinement residual in full (no residual update).
 */
enum { CTR_FARFIELD_DIRECT = 0, CTR_FARFIELD_TREECODE = 1 };

/*
 * How a CTR_FP32_REFINE solve forms the residuals of its refinement steps
 * (x_{k+1} = x_k + d_k, d_k from an FP32-operator GMRES solve of A d = r_k):
 *   CTR_RESIDUAL_UPDATE  r_1 = g - A x_1 in the residual arithmetic (opt.residual);
 *       every later r_{k+1} = r_k - A d_k with the FP32-pair operator, once
 *       |r_k| <= 1e-4 |g| (before that, g - A x again; always with the treecode,
 *       whose FP32 operator is also an approximation).  A is linear, so this is
 *       g - A x_{k+1} with the FP32 operator's error (about 1e-7 relative,
 *       measured) applied to the small correction d_k only: for |r_k| ~ 1e-5 |g|
 *       the residual is off by about 1e-12 |g|.  One application of the
 *       FP64-accurate operator per solve instead of one per refinement step.
 *   CTR_RESIDUAL_FULL    every r_k = g - A x_k in the residual arithmetic.
 */
enum { CTR_RESIDUAL_UPDATE = 0, CTR_RESIDUAL_FULL = 1 };

typedef struct {
    int64_t n[3];       /* nodes per axis (nx, ny, nz), each >= 5 */
    double origin[3];   /* coordinates of node (0, 0, 0) */
    double h;           /* grid spacing, > 0 */
} ctr_grid;

typedef struct {
    double tube_halfwidth; /* eps of the tube |d| < eps; <= 0 selects 2h (Secs. 2.5, 3.3) */
    int precision;         /* CTR_FP64, or CTR_FP32_REFINE: FP32 pair sums inside FP64 refinement */
    double tol;            /* relative residual |g - A x| / |g| to reach; <= 0 selects 1e-10 */
    int restart;           /* Krylov vectors per GMRES cycle; <= 0 selects 64 */
    int max_iter;          /* limit on GMRES iterations (all cycles, all refinements); <= 0: 400 */
    int max_refine;        /* limit on refinement steps (CTR_FP32_REFINE); <= 0 selects 10 */
    double inner_tol;      /* relative tolerance of each FP32 GMRES solve; <= 0 selects 1e-5 */
    int tile_targets;      /* reserved, ignored */
    int residual;          /* pair arithmetic of the refinement residual r = g - A x:
                              CTR_DF64 (the default of ctr_default_options) or CTR_FP64 */
    int method;            /* CTR_METHOD_HYB (default) or CTR_METHOD_KREG */
    int farfield;          /* CTR_FARFIELD_DIRECT (default) or CTR_FARFIELD_TREECODE */
    int tree_degree;       /* treecode interpolation degree per axis, 2..12; <= 0 selects 10 */
    double tree_theta;     /* treecode separation parameter, 0 < theta < 1; <= 0 selects 0.8 */
    int tree_leaf;         /* most nodes of a treecode leaf; <= 0 selects 128 */
    int tree_degree_fp32;  /* degree of the CTR_FP32_REFINE operator (the inner GMRES, whose own
                              rounding is ~2e-5); <= 0 selects 6 */
    double tree_theta_fp32;/* theta of the CTR_FP32_REFINE operator; <= 0 selects 0.9 */
    int residual_mode;     /* CTR_RESIDUAL_UPDATE (default) or CTR_RESIDUAL_FULL (see above) */
    int fp32_block;        /* targets per block of the FP32 pair kernel, 512 or 1024; 0: tuned */
    int fp32_tile;         /* sources per shared-memory tile of the FP32 pair kernel, 128 or 256; 0: tuned.
                              With both 0 the setup picks the FP32 kernel variant (block, tile,
                              transposed chunk, unroll) by timing every variant on the system itself,
                              once per device and size bucket (floor(log2 M)) per process, and keeps
                              the choice for later systems of that bucket (see ctr_ibim_pair_tuning).
                              Block and tile fix the FP32 summation order, so a system's results are
                              the same alone and in any batch of the process; another process may
                              time differently and choose another variant (results then differ
                              within the FP32 operator's rounding).  Treecode handles use 1024, 256. */
} ctr_options;

typedef struct {
    int64_t iterations;    /* GMRES iterations, all cycles and refinements */
    int64_t refinements;   /* refinement steps (FP64-accurate residual evaluations) */
    int64_t matvecs_fp32;  /* FP32-pair operator applications (GMRES and residual updates) */
    int64_t matvecs_fp64;  /* FP64-accurate (CTR_FP64 or CTR_DF64) operator applications */
    double residual;       /* final |g - A x| / |g|: with the FP64-accurate operator, or, after a
                              residual update (CTR_RESIDUAL_UPDATE), the updated residual */
    int converged;         /* 1 when residual <= tol */
} ctr_solve_info;

typedef struct ctr_ibim ctr_ibim;

/* Fills *opt with the defaults described in ctr_options. */
void ctr_default_options(ctr_options* opt);

/*
 * Builds the discrete system for one surface and one set of charges.
 * Steps, all on the GPU: tube nodes |d| < eps (Eq. 2.4); finite-difference
 * normals, closest points P = y - d n, principal curvatures and directions,
 * Jacobian J and weights W = J delta_eps(d) (Sec. 2.1, Eqs. 2.6-2.8, phi of
 * Sec. 2.6); correction nodes and weights omega^(ij) (Sec. 2.4, Eqs.
 * 2.19-2.29); right-hand side g (Eq. 2.12).
 *   grid       grid description (host struct).
 *   sdist      signed distance, nx*ny*nz doubles, positive outside; host
 *              memory, or device memory when sdist_on_device != 0.
 *   eps_in, eps_out  dielectric constants inside / outside (> 0).
 *   kappa      screening parameter (>= 0), 1/Angstrom.
 *   n_charges  number of point charges (>= 0); charge_xyz holds 3*n_charges
 *              doubles (x, y, z per charge), charge_q n_charges doubles; host.
 *   opt        options, or NULL for the defaults.
 *   stream     cudaStream_t to run on (NULL: the legacy default stream).
 *   out        receives the handle; set to NULL on failure.
 * Errors: CTR_ERR_INVALID, CTR_ERR_EMPTY_TUBE, CTR_ERR_GRID_MARGIN,
 * CTR_ERR_NUMERIC (a non-finite signed-distance value anywhere in the grid, a
 * non-finite charge position or value, or non-finite geometry), CTR_ERR_NOMEM,
 * CTR_ERR_CUDA.
 */
int ctr_ibim_setup(const ctr_grid* grid, const double* sdist, int sdist_on_device,
                   double eps_in, double eps_out, double kappa,
                   int64_t n_charges, const double* charge_xyz, const double* charge_q,
                   const ctr_options* opt, void* stream, ctr_ibim** out);

/* Releases every device and host resource of the handle (NULL is ignored). */
void ctr_ibim_destroy(ctr_ibim* sys);

/* Number of tube nodes M (the system has 2M unknowns). */
int ctr_ibim_num_nodes(const ctr_ibim* sys, int64_t* M);

/* Grid linear index of each tube node: M int64 values, host memory. */
int ctr_ibim_nodes(const ctr_ibim* sys, int64_t* grid_index);

/*
 * Node geometry (Sec. 2.1), host memory: P (3M, x y z per node), normal
 * (3M), W = J delta_eps(d) (M).  Any pointer may be NULL to skip it.
 */
int ctr_ibim_geometry(const ctr_ibim* sys, double* P, double* normal, double* W);

/* Number of correction entries E = sum over targets of |N_h(y_i)| (Eq. 2.14). */
int ctr_ibim_num_corrections(const ctr_ibim* sys, int64_t* E);

/*
 * Correction matrix Omega of Eq. (2.30) in CSR form by target, host memory:
 * ptr (M+1 int64), node (E int64), omega11, omega12, omega21, omega22 (E
 * doubles each).  Row i adds sum_e W_m (h^2 omega11 rho1_m - h^3 omega12 rho2_m)
 * and sum_e W_m (h^2 omega21 rho1_m - h^2 omega22 rho2_m).  CTR2 rows: one
 * entry per corrected plane in ascending plane order, omega12 = kappa/(4 pi)
 * (Theorem of Sec. 2.4.1).  K-reg rows (bad targets): the nodes of the
 * tangent-plane cylinder of radius 2h in ascending node order, omega11 =
 * omega21 = omega22 = 0, omega12 = C12 of Sec. 2.3.  Any output may be NULL.
 */
int ctr_ibim_corrections(const ctr_ibim* sys, int64_t* ptr, int64_t* node, double* omega11,
                         double* omega12, double* omega21, double* omega22);

/* Hybrid classification (Sec. 3.2): flags[i] = 1 when node i is bad; M bytes, host. */
int ctr_ibim_bad_nodes(const ctr_ibim* sys, uint8_t* flags);

/* Right-hand side g = [g1; g2] of Eq. (2.12) at the nodes' P: 2M doubles. */
int ctr_ibim_rhs(const ctr_ibim* sys, double* g, int on_device);

/* Surface area by the tube rule, Eq. (2.6) with f = 1: h^3 sum_j W_j. */
int ctr_ibim_area(const ctr_ibim* sys, double* area);

/*
 * The pair schedule of one arithmetic (precision CTR_FP32_REFINE, CTR_DF64 or
 * CTR_FP64) of the dense sum of Eq. (2.30): how many (target, source) pairs
 * its one-sided items evaluate (the near band, correction pairs masked), how
 * many its symmetric items evaluate once for both orientations (each counts
 * once here and stands for two of the M^2 - |N| interactions), its work items
 * and the bytes of the device buffer its items add their sums into (exact
 * per-node accumulators, 200 bytes per node, shared by the three
 * arithmetics; the sums do not depend on the order of the additions).  Any
 * output may be NULL.
 */
int ctr_ibim_pair_schedule(const ctr_ibim* sys, int precision, int64_t* one_sided_pairs,
                           int64_t* symmetric_pairs, int64_t* items, int64_t* partial_bytes);

/*
 * The treecode of a handle set up with farfield = CTR_FARFIELD_TREECODE, for
 * one arithmetic (precision; its target blocks are 1024 tree positions for
 * CTR_FP32_REFINE and 256 for CTR_DF64 and CTR_FP64).  Outputs (host, any may
 * be NULL): perm, M int64, the node at each tree position; near_pairs, the
 * (target, source) pairs summed directly (correction pairs included in the
 * count, skipped in the sum); far_evaluations, targets x proxy points of
 * their far clusters; far_interactions, (target block, far cluster) pairs;
 * far_clusters, clusters that carry charges.  CTR_ERR_INVALID for a handle
 * without the treecode.
 */
int ctr_ibim_farfield_info(const ctr_ibim* sys, int precision, int64_t* perm, int64_t* near_pairs,
                           int64_t* far_evaluations, int64_t* far_interactions, int64_t* far_clusters);

/*
 * Profiling: `reps` applications of the operator of Eq. (2.30) in arithmetic
 * `precision` to the right-hand side g (after one untimed application), timed
 * with CUDA events on the handle's stream; the mean milliseconds of the
 * phases: packing the source weights, the pair items (the whole dense sum, or
 * the treecode's direct part), the treecode's far field (moments, charges,
 * far items; 0 without the treecode) and the finish (correction, diagonal,
 * partial sums).  Any output may be NULL.
 */
int ctr_ibim_time_operator(ctr_ibim* sys, int precision, int reps, double* pack_ms, double* pairs_ms,
                           double* far_ms, double* finish_ms);

/*
 * The tree and interaction lists of the treecode (CTR_FARFIELD_TREECODE) as a
 * host computation (no GPU): M nodes with integer grid indices ijk (3 int32
 * per node), their correction sets in CSR form over the node order (excl_ptr
 * M + 1 int32, excl int32), the box widening `margin` in grid units
 * (ceil(eps/h)), degree (2..12), theta (0 <= theta < 1; 0 makes every pair
 * direct), leaf (>= 1), target block size (>= 1) and min_far, the node count a
 * well-separated cluster must exceed to be approximated (<= 0 selects
 * (degree+1)^3; a handle uses (degree+1)^3 for its FP32 and FP64 blocks and
 * (degree+1)^3 / 2 for its float-float blocks).  Outputs (host, any may
 * be NULL): perm (M), n_near_ranges, n_far, near_ptr (nb + 1 with
 * nb = ceil(M / block)), near_rng (2 per range: [begin, end) tree positions),
 * far_ptr (nb + 1), far_begin and far_end (n_far each: the position range of
 * each far cluster).  Call with the array outputs NULL to learn the sizes.
 * CTR_ERR_INVALID, before anything is built, when an index lies outside
 * (-2^30, 2^30), excl_ptr[0] != 0, excl_ptr decreases, or an excluded node
 * lies outside [0, M).
 */
int ctr_farfield_plan(int64_t M, const int32_t* ijk, const int32_t* excl_ptr, const int32_t* excl, int margin,
                      int degree, double theta, int leaf, int block, int64_t min_far, int64_t* perm,
                      int64_t* n_near_ranges,
                      int64_t* n_far, int64_t* near_ptr, int64_t* near_rng, int64_t* far_ptr,
                      int64_t* far_begin, int64_t* far_end);

/*
 * y = A x for the operator of Eq. (2.30) (rows of Eqs. 2.14-2.15): the
 * punctured dense kernel sum, the sparse correction and the diagonal.
 *   x, y       2M doubles each ([rho1; rho2]); host or device (on_device).
 *   precision  CTR_FP64, CTR_FP32_REFINE or CTR_DF64 (see above): the
 *              arithmetic of the pair sums; the correction and the diagonal
 *              are FP64 in every case.
 */
int ctr_ibim_matvec(ctr_ibim* sys, const double* x, double* y, int precision, int on_device);

/*
 * Solves A p = g (Eq. 2.30) by GMRES (Sec. 2.5), x0 = 0, right-preconditioned
 * by the diagonal Lambda.  With CTR_FP64 (or CTR_DF64) the operator uses that
 * pair arithmetic throughout; with CTR_FP32_REFINE each GMRES solve uses the
 * FP32-pair operator inside a refinement loop whose residual r = g - A x uses
 * the pair arithmetic opt.residual (CTR_DF64 or CTR_FP64).  Vectors,
 * orthogonalisation and Givens rotations are FP64.
 *   psi, dpsi_n  M doubles each (rho1, rho2); host or device (on_device).
 *   info         may be NULL.
 * Returns CTR_NOT_CONVERGED when the iteration limits stop it first.
 */
int ctr_ibim_solve(ctr_ibim* sys, double* psi, double* dpsi_n, int on_device, ctr_solve_info* info);

/*
 * Solves n systems together (Sec. 2.5 solver, as ctr_ibim_solve, for each):
 * one multi-slot engine advances all of them in lockstep steps, each step one
 * Arnoldi iteration for every system still iterating and one true-residual
 * evaluation for every system at the end of a cycle; the dense pair sums of
 * all systems run in shared persistent launches, and the step's kernel
 * sequence is replayed as one CUDA graph.  Every system's arithmetic is the
 * same as when it is solved alone, so its result is bitwise identical.
 *   systems   n distinct handles on one device (any sizes, any options).
 *   psi, dpsi_n  n output pointers each, M_i doubles, host or device (on_device).
 *   infos     n entries, or NULL.
 * Returns CTR_NOT_CONVERGED when any system stopped at its limits.
 */
int ctr_ibim_batch_solve(ctr_ibim* const* systems, int64_t n, double* const* psi, double* const* dpsi_n,
                         int on_device, ctr_solve_info* infos);

/* ---------------------------------------------------------------- serving
 * A server solves requests (one surface + charges each) as they arrive, with
 * continuous batching: a setup thread takes waiting requests (first come,
 * first served) while a slot is free and the device-memory budget allows, and
 * sets them up on the GPU alongside the running work; a worker thread puts
 * set-up systems into free slots of one multi-slot engine, advances every
 * admitted system one engine step at a time, and retires finished ones
 * (their result and polarization energy kept until released).  Requests that
 * arrive while others run share the same launches.  Every system's
 * arithmetic is the same as when it is solved alone.  The server uses the
 * device current at ctr_server_create.
 */
typedef struct ctr_server ctr_server;

typedef struct {
    int max_slots;             /* systems resident at once, 1..4096 (default 16) */
    int64_t hbm_budget_bytes;  /* device memory the resident systems may hold; <= 0: 80% of free memory */
    /* Size of the parts of a large operator application, in milliseconds at the GPU's estimated
     * pair rate (default 20; 0: never split).  A system whose application would take longer runs it
     * in parts over consecutive engine steps (at most 127, each a balanced set of its schedule's
     * items, at least 64 items and twice the longest item's time each).  In every step such a system
     * runs one part, or as many as fit in the pair work of all other systems in that step: small
     * systems are not held back for a large system's whole application, and a large system keeps
     * about half of a busy step.  The node accumulators are exact, so the result does not depend
     * on the split.  Must be finite and in [0, 1e6]; CTR_ERR_INVALID otherwise. */
    double step_quantum_ms;
} ctr_server_options;

typedef struct {
    int status;                /* CTR_OK, CTR_NOT_CONVERGED, or a negative status of setup/solve */
    int64_t M;                 /* tube nodes of the request */
    double G_pol;              /* polarization energy, Eq. (3.3) */
    ctr_solve_info info;
    double t_submit, t_admit, t_done;   /* seconds on the server's steady clock */
} ctr_request_result;

typedef struct {
    int64_t budget_bytes, used_bytes, peak_used_bytes;
    int peak_slots, running, waiting;   /* waiting: not yet in an engine slot (queued, in setup, set up) */
    int64_t steps;
} ctr_server_stats_t;

void ctr_default_server_options(ctr_server_options* opt);
/* Starts a server (and its worker thread) on the current device. */
int ctr_server_create(const ctr_server_options* opt, ctr_server** out);
/* Queues a request; all inputs are host memory and are copied (same meaning as ctr_ibim_setup). */
int ctr_server_submit(ctr_server* sv, const ctr_grid* grid, const double* sdist, double eps_in, double eps_out,
                      double kappa, int64_t n_charges, const double* charge_xyz, const double* charge_q,
                      const ctr_options* opt, uint64_t* ticket);
/* Non-blocking: *done = 1 and *res filled once the request has finished. */
int ctr_server_poll(ctr_server* sv, uint64_t ticket, int* done, ctr_request_result* res);
/* Blocks until the request has finished (timeout_s <= 0: no limit; else CTR_ERR_DEVICE_WAIT on timeout). */
int ctr_server_wait(ctr_server* sv, uint64_t ticket, double timeout_s, ctr_request_result* res);
/* Copies a finished request's psi and dpsi_n (M doubles each, host; capacity >= M). */
int ctr_server_fetch(ctr_server* sv, uint64_t ticket, double* psi, double* dpsi_n, int64_t capacity);
/* Forgets a finished request and its stored result. */
int ctr_server_release(ctr_server* sv, uint64_t ticket);
int ctr_server_stats(ctr_server* sv, ctr_server_stats_t* out);
/*
 * Cancels a request that has not finished: a queued one leaves the queue, one
 * in setup is dropped when its setup ends, a running one leaves its engine
 * slot between two engine steps (the other systems go on unaffected).  The
 * request then finishes with status CTR_ERR_CANCELLED and no result (wait,
 * poll and release work as for any finished request).  Returns
 * CTR_ERR_INVALID for an unknown ticket or a request that has already
 * finished.
 */
int ctr_server_cancel(ctr_server* sv, uint64_t ticket);
/* Stops the server's threads (waiting requests are dropped) and frees everything. */
void ctr_server_destroy(ctr_server* sv);

/*
 * Reaction potential at every charge (Eq. 2.31, trapezoidal rule on the
 * tube) and the polarization energy G_pol = 1/2 sum_k q_k psi_rxn(z_k)
 * (Eq. 3.3).  psi, dpsi_n: M doubles each (host or device, on_device);
 * G_pol: host double; psi_rxn: n_charges host doubles or NULL.
 */
int ctr_ibim_energy(ctr_ibim* sys, const double* psi, const double* dpsi_n, int on_device,
                    double* G_pol, double* psi_rxn);

/*
 * psi_rxn of Eq. (2.31) at arbitrary points z (away from the surface), in
 * FP64: n_points points, xyz 3*n_points doubles (host), out n_points doubles
 * (host); psi, dpsi_n host or device (on_device).  The same tiled kernel as
 * ctr_ibim_potential_map with precision CTR_FP64.
 */
int ctr_ibim_reaction_potential(ctr_ibim* sys, const double* psi, const double* dpsi_n, int on_device,
                                int64_t n_points, const double* xyz, double* out);

/*
 * Potential map: psi_rxn of Eq. (2.31) (the trapezoidal rule on the tube,
 * valid at points away from the surface) at n_points arbitrary points, as a
 * tiled pair sum of the points against the M tube nodes.
 *   psi, dpsi_n  M doubles each (a solution of ctr_ibim_solve).
 *   xyz          3*n_points doubles (x, y, z per point).
 *   out          n_points doubles.
 *   precision    CTR_FP32_REFINE: FP32 pair terms, two points per f32x2
 *                instruction, per-tile sums added in FP64 (about 1e-7
 *                relative); CTR_DF64: float-float terms (about 1e-13);
 *                CTR_FP64: IEEE FP64.
 *   on_device    0: every array is host memory; 1: every array is device
 *                memory of the handle's device.
 * The split partial sums (and, for host arrays, device copies of the
 * arguments) live in buffers the handle keeps: a call allocates only when it
 * needs more than an earlier call did.  The handle's packed source weights
 * are overwritten (as by ctr_ibim_matvec).  Errors: CTR_ERR_INVALID,
 * CTR_ERR_CAPACITY (n_points >= 2^31), CTR_ERR_NOMEM, CTR_ERR_CUDA,
 * CTR_ERR_DEVICE_WAIT.
 */
int ctr_ibim_potential_map(ctr_ibim* sys, const double* psi, const double* dpsi_n, int64_t n_points,
                           const double* xyz, double* out, int precision, int on_device);

/*
 * The correction-weight tables of Sec. 2.4.2 as this library computes them
 * (Ewald summation of the limit of Eq. 2.29): out holds
 * 2 * 9 * 39 * 39 doubles, [kind][mode][ia][ib], kind 0 = |y|^-1 cos(k psi),
 * kind 1 = |y|^-1 sin(k psi), k = 0, 2, ..., 16, shift (ia - 19)/32 and
 * (ib - 19)/32.  Host memory.  Runs on the current device's default stream.
 */
int ctr_weight_tables(double* out);

/*
 * Allocation-free variant of the FP32 dense pair sum (the paper has no
 * counterpart: it is an interface for callers, not a step of the method).
 * For callers that cannot call cudaMalloc -- code running under an allocator
 * that owns all of the device's memory (a framework's caching pool, an
 * embedding application that reserved the GPU for itself), or a real-time
 * loop that must not stall on an allocation -- this entry point takes every
 * input and output from the caller and keeps its scratch (the per-split
 * partial sums) in a fixed device array of 2 * CTR_STATIC_SCRATCH_NODES
 * doubles (16 MiB), which each GPU that loads the library holds until the
 * process exits.  It calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *   M          nodes, 1 <= M <= CTR_STATIC_SCRATCH_NODES (else CTR_ERR_CAPACITY).
 *   src        device, 16-byte aligned, 8 M floats: node j is
 *              {Px, Py, Pz, a, nx, ny, nz, b} with a = h^3 W_j rho1_j / (4 pi),
 *              b = h^3 W_j rho2_j / (4 pi).
 *   row_ptr    device, M + 1 int32; excluded: device int32, for row i the
 *              ascending node ids row_ptr[i] .. row_ptr[i+1]-1 omitted from
 *              its sum (the correction nodes N(i)).
 *   eps_ratio  eps_out / eps_in;  kappa  screening parameter (>= 0).
 *   out        device, 2 M doubles: out[i] = sum_{j not excluded} (a_j 4pi K11 -
 *              b_j 4pi K12), out[M + i] = sum (a_j 4pi K21 - b_j 4pi K22), the
 *              same numbers ctr_ibim_matvec adds before the correction and
 *              the diagonal (FP32 pair terms, FP64 tile sums).
 *   stream     cudaStream_t (NULL: legacy default stream); the call returns
 *              after the stream has finished its work.
 * The first call on a device looks up that device's array address
 * (cudaGetSymbolAddress, with the device current); make that first call
 * before any stream capture.  Every call shares the array, which keeps the
 * last call's contents; calls that overlap on the GPU race on it.
 */
#define CTR_STATIC_SCRATCH_NODES 1048576
int ctr_pair_sum_fp32_static(int64_t M, const float* src, const int32_t* row_ptr, const int32_t* excluded,
                             double eps_ratio, double kappa, double* out, void* stream);

/*
 * Diagnostic: the number of polls after which the pair kernels give up
 * waiting for a source tile's bulk copy (default 2^22; polls < 0 restores
 * it).  On giving up, a block sets the handle's error word, lets the copies
 * it has in flight land, and returns; the call then fails with
 * CTR_ERR_DEVICE_WAIT and its outputs are not usable, while the device and
 * the handle stay usable.  A limit of 0 makes every wait give up at once,
 * which exercises that path without any fault.  Applies to the operator
 * applications and solves that start after the call, in every thread.
 */
int ctr_set_wait_limit(int64_t polls);

/* Status code -> short description (static string). */
const char* ctr_status_string(int status);

/* Message of the last failure on the calling thread ("" if none). */
const char* ctr_last_error(void);

/* Kernels this library has launched in this process so far (all devices and handles). */
int64_t ctr_kernel_launches(void);

/*
 * The FP32 pair-kernel variant the most recent setup in this process took from
 * its tuning (timed, or from the tuning cache; see ctr_options.fp32_block):
 * targets per thread (2 or 4), sources
 * per transposed chunk of the symmetric items (4 or 8) and unroll of the
 * chunk loop (1 or 2); all 0 before the first tuning.
 */
int ctr_tuning_info(int* targets_per_thread, int* chunk, int* unroll);

/*
 * The pair-kernel shape of one arithmetic (precision) of a handle's schedule:
 * targets per block, sources per shared-memory tile, sources per transposed
 * chunk and unroll of the chunk loop (outputs may be NULL).  CTR_FP32_REFINE:
 * the tuned or requested variant; CTR_DF64: 256, 128, 8, 1 and CTR_FP64:
 * 256, 128, 8, 1 (fixed).
 */
int ctr_ibim_pair_tuning(const ctr_ibim* sys, int precision, int* block_targets, int* tile, int* chunk,
                         int* unroll);

#ifdef __cplusplus
}
#endif

#endif /* CTR_IBIM_H */
