/*
 * mlq.h -- C ABI of libmlq, a GB300 (sm_103a) implementation of the batched
 * per-sample forward solve inside multilevel quadrature for the stochastic
 * monodomain equation (Ben Bader, Harbrecht, Krause, Multerer, Quaglino,
 * Schmidlin, "Space-time multilevel quadrature methods and their application
 * for cardiac electrophysiology", arXiv 2105.02007).
 *
 * Conventions for every call:
 *   - Every function returns an mlq_status (0 = MLQ_OK, negative = error);
 *     mlq_strerror() gives a message.  No exception or exit() crosses the ABI.
 *   - Host arrays are owned by the caller and only read (or written, for
 *     outputs) during the call; the library copies what it keeps.
 *   - Arrays documented as "host or device" may be either; the library asks
 *     the CUDA driver which one a pointer is.  Device pointers must be on the
 *     context's device; the caller keeps ownership.
 *   - A context may be shared by host threads: the calls that use the device
 *     or the level table take the context's lock (one at a time);
 *     mlq_submit / mlq_poll only touch the serving queue.
 *   - Per-sample failures (iteration cap, NaN/Inf) come back in status[] and
 *     never abort the other samples of a batch.
 *
 * Mesh convention (structured, shared with callers that build Phi tables):
 *   2D, unit square, m x m nodes: node (i,j) = i + m*j at (i/(m-1), j/(m-1));
 *   square (i,j), c = i + (m-1)*j, holds element 2c   = (i,j)(i+1,j)(i+1,j+1)
 *                                      and element 2c+1 = (i,j)(i+1,j+1)(i,j+1).
 *   Red refinement maps the m-node mesh to the (2m-1)-node mesh: the levels
 *   are nested (Sec. 3.1 of the paper: nested meshes with h_l ~ 2^-l).
 *   3D, box [0,Lx] x [0,Ly] x [0,Lz] (default 1 x 1 x 0.25), mx x my x mz
 *   nodes: node (i,j,k) = i + mx*(j + my*k) at (Lx i/(mx-1), ...); cube
 *   c = i + (mx-1)*(j + (my-1)*k) holds the six Kuhn tetrahedra 6c + s,
 *   s = 0..5, each the path from corner (i,j,k) to (i+1,j+1,k+1) stepping
 *   along the axes in the order (x,y,z), (x,z,y), (y,x,z), (y,z,x), (z,x,y),
 *   (z,y,x); the fibre direction is in-plane, f = (cos t, sin t, 0).  Regular
 *   refinement (2m-1 nodes per axis) nests these meshes.
 */
#ifndef MLQ_H
#define MLQ_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct mlq_ctx mlq_ctx; /* opaque; owns the device state it allocates */

typedef enum {
    MLQ_OK = 0,
    MLQ_EINVAL = -1,       /* bad argument (null pointer, size, unknown level) */
    MLQ_ENOMEM = -2,       /* device or host allocation failed */
    MLQ_ECUDA = -3,        /* a CUDA runtime call failed; see mlq_last_cuda_error */
    MLQ_ENOTREADY = -4,    /* serving: the request has not finished */
    MLQ_ETIMEOUT = -5,     /* a bounded wait ran out */
    MLQ_EUNSUPPORTED = -6, /* valid request this build does not implement */
    MLQ_ETOOBIG = -7       /* request larger than mlq_solve_noalloc's fixed scratch */
} mlq_status;

typedef enum { MLQ_FP64 = 0, MLQ_MIXED = 1 } mlq_precision;

/* per-sample outcome written to status[] */
typedef enum {
    MLQ_S_CONVERGED = 0, /* every time block reached its tolerance */
    MLQ_S_MAXITER = 1,   /* some block hit max_iter (the sample still finished) */
    MLQ_S_NONFINITE = 2, /* NaN/Inf met: the sample stopped, its QoI is NaN */
    MLQ_S_CANCELLED = 3
} mlq_sample_status;

/* Monodomain model with FitzHugh-Nagumo kinetics (eq. monodomain and
 * eq. ionic_term; the two-variable nondimensional form):
 *   dv/dt - div(D grad v) = v (v - a)(1 - v) - w,   dw/dt = eps (v - gamma w),
 *   D = s_t I + (s_l - s_t) f f^T,  f = (cos t, sin t)             (eq. AdmV)
 * with homogeneous Neumann boundary conditions on [0, T].
 * Defaults: s_l 1.0, s_t 0.2, a 0.1, eps 0.01, gamma 0.5, T 10. */
typedef struct {
    double s_l, s_t, a, eps, gamma, T;
} mlq_model;

/* Solver options.
 *   precision  MLQ_FP64: FP64 Jacobi-PCG per time block, stopping at
 *                        ||r|| <= rtol ||b||.
 *              MLQ_MIXED: FP32 Jacobi-PCG (FP32 stencil apply and vector
 *                        updates, FP64 cross-thread dot sums) inside an FP64
 *                        iterative-refinement loop whose FP64 residual stops
 *                        at ||b - A v|| <= rtol ||b||; each FP32 solve stops
 *                        at rtol_inner times its starting residual.
 *   max_iter   cap on CG iterations per solve (per refinement sweep).
 *   max_sweeps cap on refinement sweeps per block (MLQ_MIXED only).
 *   cluster    CTAs per sample (1,2,4,6,8,12,16; 2D levels take 6 as 4 and
 *              12 as 8); 0 = chosen per level.
 *   threads    threads per CTA (64..512, multiple of 32; 3D levels use at
 *              most 256); 0 = chosen.
 *   storage    where a sample's PCG vectors live: 0 = on chip (registers and
 *              shared memory of its cluster) when they fit, else global
 *              memory; 1 = on chip (a solve whose level does not fit returns
 *              MLQ_EUNSUPPORTED); 2 = global memory.
 *   graphs     1 = mlq_estimate captures its whole multi-stream launch
 *              sequence into a CUDA graph and replays it while the
 *              configuration, sizes and pointers are unchanged (needs a
 *              non-NULL stream in mlq_create and device xi / y arrays;
 *              otherwise it runs eagerly).  0 = always eager.
 *   precond    preconditioner of the inner PCG in the mixed path: 0 = Jacobi,
 *              1 = geometric multigrid V(1,1) on the nested hierarchy of the
 *              level's mesh (Galerkin coarse operators, damped Jacobi
 *              smoothing), distributed over the sample's cluster; used when
 *              its shared-memory layout fits, else Jacobi.  The FP64 path
 *              always uses Jacobi (the oracle's preconditioner). */
typedef struct {
    int precision;
    double rtol;
    double rtol_inner;
    int max_iter;
    int max_sweeps;
    int cluster;
    int threads;
    int storage;
    int graphs;
    int precond;
} mlq_options;

/* Time scheme and ionic model.
 *   ionic 0  (the default): the two-variable FitzHugh-Nagumo model of
 *            mlq_model, backward Euler for the diffusion, the reaction
 *            explicit per block (every block matrix M + dt K is SPD).
 *   ionic 1  the paper's scheme (Sec. 3.1 eq. st-system with the reaction of
 *            eq. mono_disc on the new time level): per block
 *              (M + theta dt K) u + dt M I_ion(u)
 *                = (M - (1 - theta) dt K) u_k + dt M (theta g(t_{k+1}) + (1 - theta) g(t_k)),
 *            I_ion(u) = alpha (u - u_rest)(u - u_th)(u - u_peak) (eq. ionic_term),
 *            g the nodal values of the stimulus I_app(x, t) = (u_rest + amp
 *            exp(-|x - x0|^2 / sigma^2)) for 0 <= t < t1 (Sec. 5.1);
 *            theta = 1/2 is Crank-Nicolson, 1 backward Euler.  The nonlinear
 *            block system is solved by chord-Newton sweeps (the FP64 residual
 *            of the iterate, CG on M + theta dt K for the correction) to
 *            ||F|| <= rtol ||rhs||, in both precisions; the start is u_rest
 *            unless mlq_set_initial_state gives one.  2D levels only
 *            (MLQ_EUNSUPPORTED with 3D levels); runs in the generic slab
 *            kernel (Jacobi inner preconditioner).  s_l, s_t come from
 *            mlq_model.
 * mlq_default_scheme: ionic 0, theta 1, and the paper's constants alpha
 * 1.4e-3, u_rest 0, u_th 28, u_peak 115, amp 115, t1 0.005, with sigma 0.1
 * and x0 the origin (the paper leaves sigma and x0 to the geometry). */
typedef struct {
    int ionic;
    double theta;
    double alpha, u_rest, u_th, u_peak;
    double amp, sigma, t1;
    double x0[3];
} mlq_scheme;
int mlq_default_scheme(mlq_scheme *sc);
int mlq_set_scheme(mlq_ctx *ctx, const mlq_scheme *sc);

/* Fill *opt / *model with the defaults listed above (rtol 1e-13 for FP64,
 * rtol 1e-12 and rtol_inner 1e-5 for MIXED, max_iter 100000, max_sweeps 20,
 * precond 1 (multigrid) for MIXED and 0 for FP64; mlq_solve_noalloc always
 * uses the Jacobi inner preconditioner and ignores the launch options). */
int mlq_default_options(mlq_options *opt, int precision);
int mlq_default_model(mlq_model *model);

/* Create a context on CUDA device `device` issuing work on `cuda_stream`
 * (a cudaStream_t, e.g. torch.cuda.current_stream().cuda_stream; NULL = the
 * legacy default stream).  opt may be NULL (FP64 defaults). */
int mlq_create(mlq_ctx **out, int device, void *cuda_stream, const mlq_options *opt);
int mlq_destroy(mlq_ctx *ctx);
int mlq_set_options(mlq_ctx *ctx, const mlq_options *opt);
int mlq_set_model(mlq_ctx *ctx, const mlq_model *model);

/* Declare level `level` (0..15) of the nested hierarchy {T_l} (Sec. 3.1)
 * with time step dt and nsteps time blocks (nsteps dt = T):
 *   dim = 2: the m x m node mesh of the unit square (dims[0] = m, lengths
 *            ignored);
 *   dim = 3: the mx x my x mz node Kuhn mesh of the box (dims = {mx, my, mz},
 *            each >= 2, at most 2^27 nodes; lengths = {Lx, Ly, Lz} or NULL
 *            for 1 x 1 x 0.25).  The mixed path solves 3D levels with the
 *            vectors in device memory (one cluster per sample) and a
 *            multigrid preconditioner when every axis has an odd node count
 *            >= 3; mlq_autotune and mlq_solve_noalloc are 2D only. */
int mlq_add_level(mlq_ctx *ctx, int level, int dim, const int32_t *dims, const double *lengths, double dt,
                  int32_t nsteps);

/* A level on a general tetrahedral mesh (the non-nested hierarchies of
 * Sec. 5.4, eq. PimpedML): n nodes (xyz host, n x 3), ne tetrahedra (conn
 * host, ne x 4, 0-based node indices), frames as in mlq_mesh_create (host,
 * ne x 6: the unit vectors e1, e2 of the fibre plane per tetrahedron, or
 * NULL = the x and y axes), dt and nsteps as mlq_add_level.  The level takes
 * mlq_set_kl (phi: ne x K, the modes at the tetrahedra, e.g. moved from
 * another mesh by mlq_p1_at_points), mlq_set_initial_state (n nodes) or
 * mlq_set_initial_disk (v = 1 where |x|^2 <= radius^2 over the three
 * coordinates; radius 0.1 until set), and runs in mlq_solve (the coarse
 * member of with_coarse is level - 1, structured or general, on the same xi)
 * and mlq_estimate / mlq_estimate_adaptive: a level difference Y_l =
 * Q_l - Q_{l-1} between unrelated meshes is eq. PimpedML's with both QoIs the
 * integral of v(T) on their own mesh.  Its members run the general-mesh
 * solver (as mlq_mesh_solve_opts: Jacobi-PCG, FP64 or FP32 inside FP64
 * refinement by the context's precision, rtol, rtol_inner, max_iter,
 * max_sweeps; cluster requests 6 and 12 take 4 and 8; precond, storage and
 * threads do not apply).  mlq_set_points / mlq_solve_points record the point
 * QoIs on such a level (a point's tetrahedron by the rule of
 * mlq_p1_at_points); mlq_solve_state returns its final state and
 * mlq_synthesize its KL table (FP64 in both precisions, the general-mesh
 * solver's synthesis); mlq_submit serves requests on it beside those of
 * structured levels.  mlq_autotune returns MLQ_EUNSUPPORTED on such a
 * level; the paper's time discretization (mlq_set_scheme) is for 2D levels.
 * MLQ_EINVAL for bad sizes, indices or a degenerate tetrahedron. */
int mlq_add_level_mesh(mlq_ctx *ctx, int level, int64_t n, const double *xyz, int64_t ne, const int32_t *conn,
                       const double *frames, double dt, int32_t nsteps);

/* Initial state of a level (host arrays of n nodes; w0 may be NULL = 0).
 * Without this call a level starts from v = 1 where x^2 + y^2 <= radius^2,
 * else 0, w = 0, with radius = 0.1 (mlq_set_initial_disk changes radius). */
int mlq_set_initial_state(mlq_ctx *ctx, int level, const double *v0, const double *w0);
int mlq_set_initial_disk(mlq_ctx *ctx, int level, double radius);

/* KL mode table of a level: the fibre angle on element e is
 *   theta_e = theta_mean[e] + sum_k phi[e*K + k] xi[k]         (eq. KLlowrank)
 * phi: host, n_elem x K, row-major, FP64 (n_elem from the mesh convention);
 * theta_mean: host, n_elem, may be NULL (= 0).  K <= 256.  The table holds the
 * fine-level modes transferred to this level by the midpoint rule (Sec. 4,
 * intergrid transfer): see mlq_centroid_table. */
int mlq_set_kl(mlq_ctx *ctx, int level, int K, const double *phi, const double *theta_mean);

/* Host helper: KL modes of the covariance c(x,y) = sigma2 exp(-|x-y|^2 / ell)
 * on a structured mesh (dim 2: dims[0] = m, unit square; dim 3: dims =
 * {mx, my, mz} with lengths as in mlq_add_level), by K steps of
 * pivoted Cholesky C ~ L L^T (eq. approxEig) and the reduced K x K
 * eigenproblem L^T M L v~ = lambda v~ with the P1 mass matrix M (eq. redEig).
 * modes_out: host, n x K row-major, v_k = L v~_k (so v_i^T M v_j =
 * lambda_i delta_ij), largest-magnitude entry positive; lambda_out: host, K,
 * descending. */
int mlq_build_kl(int dim, const int32_t *dims, const double *lengths, double sigma2, double ell, int K,
                 double *modes_out, double *lambda_out);

/* Host helper: midpoint-rule transfer (Sec. 4) of nodal modes on the fine
 * structured mesh (2D: fine_dims[0] = mf; 3D: fine_dims = {mx, my, mz}) to a
 * coarse nested mesh of the same domain (coarse_dims likewise):
 * phi_out[e*K + k] = fine P1 interpolant of mode k at the centroid of coarse
 * element e.  modes_f: host, n_fine x K; phi_out: host, n_elem_c x K. */
int mlq_centroid_table(int dim, const int32_t *fine_dims, const double *modes_f, int K,
                       const int32_t *coarse_dims, double *phi_out);

/* Host helper: KL modes (as mlq_build_kl, eqs. approxEig and redEig) on a
 * general simplicial mesh: xyz host, n x dim node coordinates; conn host,
 * ne x (dim + 1) node indices (0-based, each < n) of triangles (dim 2) or
 * tetrahedra (dim 3).  The P1 mass matrix is assembled from the simplices
 * (|e| (1 + delta_ab) / ((dim + 1)(dim + 2)) per simplex).  modes_out: host,
 * n x K; lambda_out: host, K, descending.  MLQ_EINVAL for a bad mesh or K
 * outside 1 .. min(n, 4096). */
int mlq_build_kl_mesh(int dim, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, double sigma2,
                      double ell, int K, double *modes_out, double *lambda_out);

/* Host helper: values at np points (pts host, np x dim) of the P1
 * interpolants of K nodal fields (f host, n x K) on a general simplicial
 * mesh (xyz, conn as in mlq_build_kl_mesh): the intergrid transfer of Sec. 4
 * between meshes that are not nested (Sec. 5.4), e.g. phi_out of a level =
 * the finest-mesh modes at that level's element centroids.  A point takes
 * the first simplex (in element order) that contains it; a point in no
 * simplex (a centroid near a curved boundary discretised differently) takes
 * the first simplex whose smallest barycentric coordinate is within 1e-12 of
 * the largest over all simplices, and the linear extension of its P1
 * function (each such point costs a scan over all simplices; points inside
 * are found through a bucket grid).  Runs on the host's cores.
 * out: host, np x K. */
int mlq_p1_at_points(int dim, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, int K, const double *f,
                     int64_t np, const double *pts, double *out);

/* mlq_p1_at_points on the current CUDA device: the same transfer and the
 * same rule (the first simplex in element order whose barycentric
 * coordinates are >= -1e-12; for a point in no simplex the first whose
 * smallest coordinate is within 1e-12 of the largest over all simplices),
 * with the bucket grid built, the points located and the fields
 * interpolated by kernels (each point outside the mesh scans every simplex
 * in a CTA of its own).  Arguments as mlq_p1_at_points (host arrays);
 * ne < 2^31.  Blocks until out is written. */
int mlq_p1_at_points_gpu(int dim, int64_t n, const double *xyz, int64_t ne, const int32_t *conn, int K,
                         const double *f, int64_t np, const double *pts, double *out);

/* Host helper: numbers of samples per level for eq. StandardML with Monte
 * Carlo rules that minimise the cost sum_l N_l cost[l] subject to the
 * statistical error sqrt(sum_l var[l] / N_l) <= eps:
 * N_l = max(nmin, ceil(eps^-2 sqrt(var[l] / cost[l]) sum_k sqrt(var[k] cost[k]))).
 * var (V_l of the level differences, >= 0), cost (> 0, e.g. DOF-steps per
 * sample) and N_out are host arrays of L + 1 entries.  MLQ_EINVAL for bad
 * arguments or counts beyond 4e18. */
int mlq_mlmc_allocation(int L, const double *var, const double *cost, double eps, int64_t nmin, int64_t *N_out);

/* Host helper: eq. StandardML (Monte Carlo rules) from per-sample level
 * differences: y[l] (host, N[l] values of Y_l = Q_l - Q_{l-1}, N[l] >= 1)
 * for l = 0..L.  mean_out = sum_l mean(Y_l); var_out[l] (may be NULL) the
 * unbiased sample variance of Y_l (0 for N[l] = 1); rmse_out (may be NULL)
 * = sqrt(sum_l var_l / N[l]).  Sums run in index order, so samples solved on
 * several processes and gathered back in index order give the same result as
 * one process, bit for bit. */
int mlq_mlmc_combine(int L, const int64_t *N, const double *const *y, double *mean_out, double *var_out,
                     double *rmse_out);

/* Host helpers for field-valued quantities of interest (the state v_h(T) of
 * mlq_solve_state) on the structured nested levels:
 * mlq_field_prolong: the P1 interpolant of a coarse field vc (coarse_dims as
 *   in mlq_add_level; n_c values) at the nodes of the nested fine mesh with
 *   2m - 1 nodes per axis (vf, n_f values): the intergrid transfer that the
 *   level differences Y_l = v_l - I v_{l-1} of eq. StandardML need for a
 *   field QoI.  Fine nodes at coarse nodes keep their value, the others take
 *   the mean of the two ends of the coarse edge they halve.
 * mlq_field_norms: ||e||_{L2(D)} and ||e||_{H1(D)} of the P1 function with
 *   nodal values e on a structured level (lengths as in mlq_add_level, NULL =
 *   the default box; ignored in 2D): the space norms of the error metric of
 *   Sec. 5 (eq. space-time-error at one time).  Either output may be NULL. */
int mlq_field_prolong(int dim, const int32_t *coarse_dims, const double *vc, double *vf);
int mlq_field_norms(int dim, const int32_t *dims, const double *lengths, const double *e, double *l2, double *h1);

/* Host helper: eq. PimpedML with nested sample rules, the multilevel
 * quadrature for levels whose meshes are not nested (Sec. 4, Sec. 5.4):
 *   est = sum_{l=0}^{L} (Q_l - Q_{l-1})(F_{L-l}),  Q_{-1} = 0,
 * Q_l the mean over the first N_l points (1 <= N_0 <= ... <= N_L).  F[l]
 * (host) holds F_{L-l}, the QoI computed on mesh L-l alone, at the first
 * N_l points; each term needs one mesh, so no transfer between the meshes
 * of different levels enters.  Sums in index order. */
int mlq_pimped_ml_combine(int L, const int64_t *N, const double *const *F, double *est_out);

/* Levels on general tetrahedral meshes (non-nested hierarchies; Sec. 4 and
 * the ventricle of Sec. 5.4): a self-contained member.  One object per
 * mesh; it owns its device arrays and uses the default stream.
 *
 * mlq_mesh_create: n nodes (xyz host, n x 3), ne tetrahedra (conn host,
 * ne x 4, 0-based, non-degenerate, ne <= 2^27), optional fibre frames
 * (frames host, ne x 6: two orthonormal vectors e1, e2 per tetrahedron; NULL
 * = the x and y axes).  Sets up the CSR pattern of the P1 matrices, the
 * element geometry and the consistent mass M (|e| (1 + delta_ab) / 20).
 * MLQ_EINVAL for bad sizes, indices or a degenerate tetrahedron.
 * mlq_mesh_set_kl: the per-element KL table phi (host, ne x K) and mean angle
 * theta_mean (host, ne, may be NULL = 0); the fibre of sample s on element e
 * is f = cos(theta) e1 + sin(theta) e2 with theta = theta_mean_e + sum_k
 * phi[e K + k] xi[s K + k] (eq. KLlowrank), D = s_t I + (s_l - s_t) f f^T
 * (eq. AdmV).
 * mlq_mesh_solve: S samples (xi host, S x K), nsteps time blocks of dt from
 * the initial state v0, w0 (host, n; w0 may be NULL = 0): b = M (v + dt R),
 * (M + dt K) v+ = b by Jacobi-preconditioned CG from v until ||b - A v+|| <=
 * rtol ||b|| (at most 10 n iterations per block), w += dt eps (v - gam w);
 * q_out (host, S) = m^T v(T) with m = M 1; status (mlq_sample_status, worst
 * block) and iters (CG iterations summed over blocks) may be NULL.  Blocks
 * until done. */
typedef struct mlq_mesh mlq_mesh;
int mlq_mesh_create(mlq_mesh **out, int device, int64_t n, const double *xyz, int64_t ne, const int32_t *conn,
                    const double *frames);
int mlq_mesh_destroy(mlq_mesh *mesh);
int mlq_mesh_set_kl(mlq_mesh *mesh, int K, const double *phi, const double *theta_mean);
int mlq_mesh_solve(mlq_mesh *mesh, const mlq_model *model, double dt, int32_t nsteps, double rtol, const double *v0,
                   const double *w0, int64_t S, const double *xi, double *q_out, int32_t *status, int32_t *iters);

/* mlq_mesh_solve with solver options (opt: precision MLQ_FP64 or MLQ_MIXED,
 * rtol, rtol_inner, max_iter per solve, max_sweeps, cluster: CTAs per
 * sample, 0 = chosen, 1, 2, 4, 8, 16 = one thread-block cluster per sample,
 * 17..4096 = that many CTAs per sample in one cooperative launch (every CTA
 * resident at once: MLQ_EUNSUPPORTED when they cannot be; their barriers
 * wait a bounded time and a wait that runs out returns MLQ_ETIMEOUT with the
 * samples' status MLQ_S_NONFINITE); the chosen shape is the cooperative one
 * when a cluster of 16 per sample would leave SMs idle and each CTA keeps
 * >= 2048 rows; the other fields are ignored).  MLQ_FP64: Jacobi-PCG in FP64 to
 * ||b - A v|| <= rtol ||b||.  MLQ_MIXED: FP32 Jacobi-PCG (FP32 CSR values and
 * vectors, FP64 sums across threads) inside FP64 iterative refinement with
 * the FP64 residual, to the same test.  The whole block loop runs in one
 * launch, one sample per cluster of CTAs (each CTA a band of CSR rows), with
 * no host synchronisation inside the solve.  mlq_mesh_solve is this call
 * with FP64 defaults, the given rtol and at most 10 n iterations per block. */
int mlq_mesh_solve_opts(mlq_mesh *mesh, const mlq_model *model, const mlq_options *opt, double dt, int32_t nsteps,
                        const double *v0, const double *w0, int64_t S, const double *xi, double *q_out,
                        int32_t *status, int32_t *iters);

/* Self-test of the barrier and sums that the cooperative launch shapes use
 * (many CTAs per sample, meeting in global memory): one cooperative launch
 * of `ctas` CTAs (1..64) on `device` through `rounds` barrier-and-sum rounds
 * (1..1000), every CTA checking the exact sum; `missing` (0..64) CTAs are
 * counted in the group but never launched, so with missing > 0 no barrier
 * completes.  Every wait gives up after `max_polls` polls (>= 1; a poll is
 * ~0.1-0.2 us): the kernel then records the time-out, returns without
 * completing, and the device stays usable.  Returns MLQ_OK (every barrier
 * completed, every sum exact), MLQ_ETIMEOUT (a wait ran out), MLQ_EINVAL
 * (bad arguments, or a wrong sum), MLQ_ECUDA / MLQ_ENOMEM. */
int mlq_group_selftest(int device, int ctas, int rounds, int missing, int64_t max_polls);

/* Solve S samples (0 <= S <= 65535) on `level`.  xi: host or device, S x K row-major FP64
 * (sample s uses xi[s*K .. s*K+K-1]).  For each sample: synthesise theta
 * (eq. KLlowrank), set up A = M + dt K(theta), run the nsteps time blocks,
 * and return the QoI Q = integral of v_h(T) = m^T v (m = M 1).
 * with_coarse != 0 also solves the same samples on level-1 (same xi) and
 * returns Y = Q_l - Q_{l-1} (eq. StandardML's level difference).
 * Outputs (host or device, FP64 / int32, length S; any may be NULL):
 *   q_fine, q_coarse, y, status (mlq_sample_status, worst of both members),
 *   iters (CG iterations summed over blocks and sweeps, fine member).
 * Blocks until the results are written. */
int mlq_solve(mlq_ctx *ctx, int level, int64_t S, const double *xi, int with_coarse, double *q_fine,
              double *q_coarse, double *y, int32_t *status, int32_t *iters);

/* The field-valued result of a solve: the state at the final time of S
 * samples (0 <= S <= 65535) on `level`, as mlq_solve computes it (same
 * kernels, same launch shape, no coarse member).  Sec. 2.4 of the paper lets
 * the QoI be a functional of the solution; this call returns the solution
 * itself, the P1 nodal values of v_h(T) and of the recovery variable w(T).
 * xi: host or device, S x K.  Outputs (host or device; any may be NULL):
 *   v_out, w_out  S x n FP64, sample-major (v_out[s*n + i], node order of
 *                 the mesh convention above; on a general-mesh level the
 *                 order of its xyz);
 *   q_out         S FP64, Q = m^T v(T) (as mlq_solve's q_fine);
 *   status        S int32 (mlq_sample_status).
 * A sample that met NaN/Inf stops early and its state is undefined.  Blocks
 * until the results are written. */
int mlq_solve_state(mlq_ctx *ctx, int level, int64_t S, const double *xi, double *v_out, double *w_out,
                    double *q_out, int32_t *status);

/* Point quantities of interest (Sec. 2.4): the action potential u(x_p, t)
 * and the activation time a(x_p) = min{t in [0, T] : u(x_p, t) >= u_th} at a
 * few points x_p of a level, formed inside the solver's block loop.
 *
 * mlq_set_points: np points (0 <= np <= 32; 0 clears) of `level`, pts host,
 * np x dim coordinates inside the level's domain (1e-12 slack), and the
 * threshold u_th.  Each point is located once: the simplex of the mesh
 * convention holding it (the first of its cell; the cell whose lower corner
 * is floor(x / h)) and its barycentric weights, so u(x_p, t) is the P1 value
 * of v_h(t) there; on a general-mesh level (mlq_add_level_mesh, dim 3) the
 * first tetrahedron of the mesh holding it (mlq_p1_at_points' rule).
 * MLQ_EINVAL for a point outside the domain (general mesh: a barycentric
 * coordinate below -1e-9 in the best tetrahedron).
 *
 * mlq_solve_points: S samples xi (host or device, S x K) on `level`, the
 * same kernels and launch shape as mlq_solve.  Outputs (host or device; any
 * may be NULL):
 *   trace   S x np x (nsteps + 1) FP64: u(x_p, t_n) at t_n = n dt, n = 0 the
 *           initial state (NaN after a sample stopped on NaN/Inf);
 *   act     S x np FP64: a(x_p), with u(x_p, .) linear in time between block
 *           ends: 0 if u(x_p, 0) >= u_th, else t_{n-1} + dt (u_th - u_{n-1}) /
 *           (u_n - u_{n-1}) at the first n with u_n >= u_th; -1 if u never
 *           reaches u_th on [0, T] (the paper's "not activated");
 *   q_out   S FP64 (Q = m^T v(T), as mlq_solve); status S int32.
 * MLQ_EINVAL if the level has no points.  Blocks until done. */
int mlq_set_points(mlq_ctx *ctx, int level, int np, const double *pts, double u_th);
int mlq_solve_points(mlq_ctx *ctx, int level, int64_t S, const double *xi, double *trace, double *act,
                     double *q_out, int32_t *status);

/* Host helpers for time quantities of interest (traces u_n at t_n = n dt,
 * read as the function linear in time between them):
 * mlq_trace_prolong: the coarse trace (nt_coarse + 1 values, step 2 dt) on the
 *   fine time grid (2 nt_coarse + 1 values): the intergrid transfer in time
 *   of Sec. 5 that the level differences of eq. StandardML need.
 * mlq_time_norms: the L2(0, T) and H1(0, T) norms (eq. point-error, q = 0,
 *   1) of the linear interpolant of e (nt + 1 values on [0, T]); either
 *   output may be NULL. */
int mlq_trace_prolong(int nt_coarse, const double *u_c, double *u_f);
int mlq_time_norms(int nt, double T, const double *e, double *l2, double *h1);

/* Multilevel Monte Carlo estimate (eq. StandardML with MC rules) over levels
 * 0..L (L <= 5): level l draws N[l] samples (2 <= N[l] <= 65535) xi[l] (host or device, N[l] x K_l) and
 * contributes the sample mean of Y_l = Q_l - Q_{l-1} (Q_{-1} = 0).  All
 * levels run concurrently.  Outputs (host): mean_out = sum_l mean(Y_l);
 * var_out[l] = unbiased sample variance of Y_l (may be NULL); rmse_out =
 * sqrt(sum_l var_l / N_l) (may be NULL); y_out[l] (host or device, N[l],
 * may be NULL or contain NULLs) the per-sample Y_l. */
int mlq_estimate(mlq_ctx *ctx, int L, const int64_t *N, const double *const *xi, double *mean_out,
                 double *var_out, double *rmse_out, double *const *y_out);

/* Adaptive multilevel Monte Carlo (eq. StandardML with the sample numbers of
 * mlq_mlmc_allocation): solve n_pilot (>= 2) samples of every level pair
 * 0..L, estimate the variances V_l of Y_l, allocate N_l for the target
 * statistical error eps with the cost of a sample of pair l taken as its
 * DOF-steps (n_l nsteps_l + n_{l-1} nsteps_{l-1}), solve the missing samples,
 * and repeat until the allocation for the latest variances is met.  xi[l]
 * (host or device, Nmax[l] x K, Nmax[l] >= n_pilot) is the pool of level l,
 * used in index order; N_l never exceeds Nmax[l] (then rmse_out may stay
 * above eps).  Outputs (host): N_out[l] the samples used, mean_out, var_out[l]
 * (may be NULL), rmse_out (may be NULL) = sqrt(sum_l V_l / N_l) over exactly
 * the samples 0..N_l-1 of each pool (as mlq_mlmc_combine).  The sample
 * numbers depend only on the values, so a rerun gives the same result.
 * MLQ_ETIMEOUT if the allocation still grew after 16 rounds. */
int mlq_estimate_adaptive(mlq_ctx *ctx, int L, double eps, int64_t n_pilot, const int64_t *Nmax,
                          const double *const *xi, int64_t *N_out, double *mean_out, double *var_out,
                          double *rmse_out);

/* The KL synthesis step alone (eq. KLlowrank), for verification: for S
 * samples xi (host or device, S x K) write cs2_out[(s*n_elem + e)*2 + {0,1}]
 * = (cos 2 theta, sin 2 theta) of element e (host or device, FP64).  The mixed
 * path computes theta on the tensor cores (tcgen05, TF32 operands split into
 * high and low parts, ~21-bit products, FP32 accumulation); the FP64 path on
 * the CUDA cores in FP64 (on a general-mesh level both paths run the
 * general-mesh solver's FP64 synthesis).  MLQ_ETIMEOUT if a bounded device
 * wait ran out. */
int mlq_synthesize(mlq_ctx *ctx, int level, int64_t S, const double *xi, double *cs2_out);

/* Bytes of device workspace a solve of S samples on `level` (and level-1
 * when with_coarse) uses; the context allocates and caches it. */
int mlq_workspace_bytes(mlq_ctx *ctx, int level, int64_t S, int with_coarse, size_t *bytes);

/* Per-member timing.  With profiling on, every solve / estimate records CUDA
 * events on the stream of each member (a level's fine or coarse batch)
 * around its slab-solver kernel; mlq_member_profile then returns, for the
 * last call, one record per member (up to max_members; *count = members of
 * that call).  The records stay valid until the next solve / estimate.
 * Profiling adds two event records per member and one small device-to-host
 * copy per member when queried. */
typedef struct {
    double kernel_ms;       /* slab-solver kernel duration (CUDA events) */
    int level, coarse;      /* level of the mesh; 1 = coarse member of a pair */
    int cluster, resident;  /* launch shape used (resident as in mlq_level_launch) */
    int threads, npt;       /* threads per CTA; nodes per thread (register kernel, else 0) */
    int64_t samples, nodes, steps;
    int64_t cg_iterations;  /* CG iterations summed over samples, blocks, sweeps */
    double start_ms, end_ms; /* kernel start / end after the start of the call (events) */
} mlq_member_stats;
int mlq_set_profiling(mlq_ctx *ctx, int enable);
int mlq_member_profile(mlq_ctx *ctx, int max_members, int *count, mlq_member_stats *out);

/* Autotuner (mixed path).  Times every register-resident launch shape of
 * `level` that fits the device (cluster size x nodes per thread) on a probe
 * run of probe_steps time blocks with the given S samples xi (host or
 * device), after one warm-up pass, and keeps the fastest for later solves of
 * this level (until the level is redefined or an explicit cluster/threads
 * option is set).  Outputs (may be NULL): chosen cluster size, threads per
 * CTA, and the probe time in milliseconds.  MLQ_EUNSUPPORTED in FP64 mode. */
int mlq_autotune(mlq_ctx *ctx, int level, int64_t S, const double *xi, int probe_steps, int *cluster_out,
                 int *threads_out, double *ms_out);

/* Solve without allocating anything.
 *
 * For callers that cannot call cudaMalloc when they need a solve: processes
 * whose device memory belongs to another allocator with a fixed budget (a
 * serving engine that reserved its HBM up front, a framework's caching
 * allocator), where a library allocation would fail or break the budget, and
 * latency-critical loops that must not take the device-wide synchronisation
 * a cudaMalloc/cudaFree may imply.  No context is needed: the call creates no
 * stream, event or buffer, and calls no cudaMalloc/cudaFree or other
 * allocating routine.
 *
 * What runs: the FP64 KL synthesis kernel (eq. KLlowrank on the CUDA cores,
 * not the tensor-core variant mlq_solve uses in the mixed path), the stencil
 * set-up, and the register-resident slab solver with the Jacobi inner
 * preconditioner, FP32 inner PCG inside FP64 refinement; one level, no coarse
 * member.  Its QoI agrees with mlq_solve (mixed path, either preconditioner)
 * within the mixed-path tolerance (1e-6 relative), not bit for bit.  The
 * launch shape is chosen by the call: opt->cluster, opt->threads,
 * opt->storage, opt->graphs and opt->precond are ignored.  All working memory
 * is one fixed, statically allocated device array of
 * MLQ_NOALLOC_SCRATCH_BYTES that every GPU which loads the library holds
 * until the process exits.  Requests whose working set does not fit return
 * MLQ_ETOOBIG; the working set is about
 *   92 * S * m^2 + 32 * S * (m-1)^2 bytes  (m x m nodes, S samples),
 * e.g. 33 x 33 nodes with up to ~250 samples, or 257 x 257 nodes with 4.
 *
 * Arguments: structured 2D level of m x m nodes, time step dt, nsteps time
 * blocks; model and opt may be NULL (defaults; opt->precision must be
 * MLQ_MIXED); K modes; phi (n_elem x K), theta_mean (n_elem or NULL), xi
 * (S x K), v0 / w0 (m^2 or NULL: the disc start of radius 0.1) -- all DEVICE
 * pointers of the current device (or managed memory), owned by the caller;
 * outputs q (S, FP64), status and iters (S, int32, may be NULL), likewise.
 * Host pointers and memory of another GPU return MLQ_EINVAL.  The work is
 * queued on cuda_stream (NULL = legacy default stream) and the call returns
 * without waiting; synchronize the stream before reading q.
 *
 * The first call on a device looks up the device address of the scratch
 * array (cudaGetSymbolAddress) with that device current.  Every call uses the same array and
 * leaves its contents behind; the kernels initialise everything they read,
 * so results do not depend on earlier calls.  Calls whose work overlaps on
 * the GPU (other streams, other host threads) race on the array: order them
 * on one stream.  (The paper has no counterpart: this is an integration
 * variant of mlq_solve.) */
#define MLQ_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)
int mlq_solve_noalloc(int m, double dt, int32_t nsteps, const mlq_model *model, const mlq_options *opt, int K,
                      const double *phi, const double *theta_mean, const double *xi, int64_t S, const double *v0,
                      const double *w0, double *q, int32_t *status, int32_t *iters, void *cuda_stream);

/* Count of kernel launches the context has issued since creation. */
int mlq_launch_count(mlq_ctx *ctx, int64_t *count);

/* Launch shape chosen for a level under the context's options: cluster size
 * (CTAs per sample), threads per CTA, and *resident: 3 = register kernel
 * with the multigrid preconditioner, 2 = the sample's PCG vectors live in
 * registers with the stencil rows in shared memory (mixed path), 1 = vectors
 * in the cluster's shared memory, 0 = in global memory.
 * resident may be NULL. */
int mlq_level_launch(mlq_ctx *ctx, int level, int *cluster, int *threads, int *resident);

/* Serving: requests for the QoI mean at one level, answered asynchronously.
 *
 * Each request asks for the plain Monte Carlo mean of Q_l (eq. SL) over at
 * most `samples` draws xi (rows of a samples x K matrix), stopping early once
 * the statistical error is small enough: the samples are solved in chunks of
 * `chunk` (a power of two), and the request finishes at the first chunk
 * boundary n where sqrt(V_n / n) <= target_rmse (V_n the unbiased sample
 * variance of the first n values, n >= 2), or after all samples.
 *
 * Continuous batching: a worker thread of the context runs up to four lanes
 * (mlq_serve_limits: 1..6),
 * each a stream with its own device workspace.  Whenever a lane is idle it
 * takes the level of the oldest waiting request whose level no lane is
 * running (one batch per level at a time, so the long batches of fine
 * levels cannot hold every lane) and packs the next chunk of every waiting
 * request at that level into one
 * batched solve (at most 2^24 DOFs and 65535 samples), so batches of
 * different levels run on the device together and a request that arrives
 * while others run starts as soon as a lane frees up.  Batches of less than
 * 1e9 DOF-steps run on high-priority streams: their CTAs take the SMs that
 * free up before those of long batches.  Lane workspaces come from the
 * device's stream-ordered memory pool, so growing one does not wait for the
 * batches of the other lanes.  A batch is admitted
 * by device memory: its lane's workspace grows only while the free HBM
 * (minus 256 MiB) and the budget of mlq_serve_limits allow it; otherwise
 * it waits for running batches, and a batch that cannot fit with every other
 * lane idle and released finishes its requests with MLQ_ENOMEM.  State stays
 * on the device for the life of a batch; between chunks a request's samples
 * wait on the host.
 *
 * Each sample's Q depends only on its own xi, and the stopping rule only on
 * the values in index order, so a request's result does not depend on what
 * it was batched with (bit for bit on the 2D levels; the launch shapes of
 * 3D and general-mesh levels follow the batch size, so there to rounding).  xi is copied at submission
 * (host pointer).  A request whose level is redefined or gets a KL table of
 * another K before it is served finishes with MLQ_EINVAL.  mlq_submit /
 * mlq_poll may be called from any thread; the worker takes the context's
 * lock only to queue a batch, so other calls run beside serving.
 * mlq_destroy stops the worker after the running batches; unfinished
 * requests are dropped. */
typedef struct {
    int level;           /* a defined level of the context */
    int64_t samples;     /* maximum number of samples, 1 .. 2^20 */
    const double *xi;    /* host, samples x K, row-major (K of the level's KL table) */
    double target_rmse;  /* <= 0: solve all samples */
    int32_t chunk;       /* samples per chunk, a power of two; 0 = 16 */
} mlq_request;

typedef struct {
    int status;            /* MLQ_OK, or the error of a batch of this request */
    int32_t worst;         /* worst per-sample status (mlq_sample_status) */
    int64_t samples_used;  /* n at which the request stopped */
    double mean, rmse;     /* mean of Q_l over the n samples and sqrt(V_n / n) */
    double latency_ms;     /* submission to completion (host clock) */
    int64_t batches;       /* batched solves the request took part in */
    double first_ms, last_ms;  /* start of its first batch and end of its last,
                                  ms after the serving worker started (host clock) */
} mlq_result;

int mlq_submit(mlq_ctx *ctx, const mlq_request *req, uint64_t *ticket);
/* Serving resources: lanes (1..6, default 4) = batches on the device at the
 * same time, each on its own stream with its own workspace; max_bytes = cap
 * on the lanes' workspaces together (0, the default: the free device memory
 * alone decides).  A batch whose workspace does not fit waits for running
 * batches; one that does not fit with every other lane idle and released
 * finishes its requests with MLQ_ENOMEM.  MLQ_ENOTREADY if lanes to be
 * dropped still run a batch (call again later). */
int mlq_serve_limits(mlq_ctx *ctx, int lanes, size_t max_bytes);
/* MLQ_ENOTREADY while the request runs; MLQ_OK fills *out and releases the
 * ticket (a second poll of it returns MLQ_EINVAL). */
int mlq_poll(mlq_ctx *ctx, uint64_t ticket, mlq_result *out);

const char *mlq_strerror(int status);
const char *mlq_last_cuda_error(mlq_ctx *ctx);

#ifdef __cplusplus
}
#endif
#endif /* MLQ_H */
