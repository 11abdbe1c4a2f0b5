/*
 * rapidnet.h -- C ABI of a GB300 (sm_103a) solver for scenario-based
 * stochastic MPC of drinking-water networks by the accelerated proximal
 * gradient method on the Fenchel dual (Sopasakis, Sampathirao, Bemporad,
 * Patrinos, "Uncertainty-aware demand management of water distribution
 * networks in deregulated energy markets", arXiv 1904.10548).
 *
 * Problem (paper §3.2, eq. SMPC): on a scenario tree with stages 0..N,
 * every non-root node nu carries an input u_nu (n_u) and a state x_nu
 * (n_x) with
 *     x_nu = A x_a(nu) + B u_nu + Gd d_nu      (eq. dynamics:tree)
 *     E u_nu + Ed d_nu = 0                     (eq. input-disturbance-coupling)
 *     umin <= u_nu <= umax                     (eq. input-constraints)
 * and the cost
 *     sum_nu p_nu [ W_alpha (alpha0 + alpha_nu)' u_nu + du' W_u du ]
 *   + sum_nu W_x dist(x_nu | [xmin, xmax]) + W_s dist(x_nu | [x_s, inf)),
 * du = u_nu - u_a(nu), with the root fixed at x_0 = p and u_{-1} = q.
 * The dual is solved by eqs. apg:1 / apg:2 (§4.3); the dual gradient is
 * a backward/forward recursion over the tree (§4.4).
 *
 * Conventions for every call:
 *   - matrices are dense, row-major, double precision, on the HOST;
 *   - nodes are numbered breadth first (node 0 = root, the nodes of stage
 *     t are [stage_ptr[t], stage_ptr[t+1]), children of a node contiguous);
 *   - per-node arrays are node-major: row nu holds node nu's vector;
 *   - the library never keeps a caller pointer past the call; what it
 *     needs is copied;
 *   - every call returns an rn_status; no call aborts, exits or throws;
 *     rapidnet_last_error() describes the last failure of this thread.
 */
#ifndef RAPIDNET_H
#define RAPIDNET_H

#ifdef __cplusplus
extern "C" {
#endif

typedef enum {
  RN_OK = 0,
  RN_NOT_CONVERGED = 1,   /* max_iters reached; outputs are valid */
  RN_ERR_INVAL = -1,      /* an argument is malformed (see last error) */
  RN_ERR_RANK = -2,       /* E does not have full row rank */
  RN_ERR_CUDA = -3,       /* a CUDA call failed */
  RN_ERR_TIMEOUT = -4,    /* a device-side wait gave up (bounded spin) */
  RN_ERR_NOMEM = -5,      /* device memory could not be obtained */
  RN_ERR_UNSUPPORTED = -6,/* valid input outside what the library handles */
  RN_ERR_DIVERGED = -7    /* the residual became NaN or infinite */
} rn_status;

typedef enum {
  RN_PREC_FP64 = 0,       /* every step of the iteration in FP64 */
  RN_PREC_MIXED = 1,      /* FP32 iteration around an FP64 reference point */
  RN_PREC_FP32 = 2        /* every step of the iteration in FP32, the factor
                             step in FP64 (per-node form only) */
} rn_precision;

/* Form of the dual gradient (rn_opts.factor_form), paper §4.4:
 *   RN_FACTOR_SHARED   the recursion collapsed onto one operator
 *                      F = W^-1 - W^-1 E'(E W^-1 E')^-1 E W^-1 shared by all
 *                      nodes, evaluated as subtree and path sums (needs
 *                      A = I; the default where it applies);
 *   RN_FACTOR_PER_NODE the general recursion with one matrix pair
 *                      (Phi_nu, K_nu) per node from the factor step,
 *                      streamed from device memory at every evaluation;
 *                      any A, nx and nu up to 1024 (FP64, also the FP64
 *                      set of RN_PREC_MIXED: while one team's vectors
 *                      and two column units fit a block's shared
 *                      memory, nx = nu up to 800; beyond it
 *                      RN_ERR_UNSUPPORTED), every precision
 *                      (RN_PREC_MIXED: FP32 matrices for the iterations and
 *                      an FP64 copy for the reference point, both on the
 *                      device); served solves (one at a time: each
 *                      launch fills the device), no batched solves, no
 *                      duality gap, no allocation-free entry point;
 *   RN_FACTOR_AUTO (0) the shared form, or the per-node form for A != I,
 *                      RN_PREC_FP32, or (RN_PREC_FP64) a layout the
 *                      shared form refuses; RN_PREC_MIXED keeps that
 *                      refusal (RN_ERR_UNSUPPORTED), which tells a batched
 *                      caller that the problem is outside solve_batch. */
enum { RN_FACTOR_AUTO = 0, RN_FACTOR_SHARED = 1, RN_FACTOR_PER_NODE = 2 };

/* Water network, paper §2.1 (eqs. dynamics, input-disturbance-coupling,
 * state-constraints, input-constraints).  Shapes: A nx*nx, B nx*nu,
 * Gd nx*nd, E ne*nu, Ed ne*nd; xmin, xmax, xs: nx; umin, umax: nu.
 * ne may be 0 (then E, Ed may be NULL).  A = I (the exact discretisation
 * of the tank mass balance, eq. tank-dynamics) is what the shared-operator
 * form handles; any other A takes the per-node form (RN_FACTOR_AUTO) or
 * gives RN_ERR_UNSUPPORTED (RN_FACTOR_SHARED). */
typedef struct {
  int nx, nu, nd, ne;
  const double *A, *B, *Gd, *E, *Ed;
  const double *xmin, *xmax, *xs, *umin, *umax;
} rn_network;

/* Scenario tree, paper §2.3 (Fig. "tree"): N stages after the root,
 * stage_ptr has N+2 entries, anc[0] = -1, anc[nu] < nu is the ancestor,
 * prob[nu] the probability of reaching nu (prob[0] = 1).  Validated: the
 * children of every node are contiguous and in parent order, their
 * probabilities sum to the parent's (relative 1e-9), every node before
 * stage N has a child, all leaves are at stage N. */
typedef struct {
  int N, n_nodes;
  const int *stage_ptr;
  const int *anc;
  const double *prob;
} rn_tree;

/* Cost weights, paper §3.1 (eqs. cost:linear, cost:smooth,
 * cost:non-smooth): W_alpha > 0, alpha0 (nu), W_u (nu*nu, symmetric
 * positive definite), W_s >= 0, W_x >= 0.  A diagonal W_u (the paper's
 * choice W_u = w I) is applied in the sparse form of the shared operator
 * F; a dense one as a dense product (tensor cores in the FP32 steps of
 * RN_PREC_MIXED), which needs chain teams of at least nu / 2 threads.
 * W_u not symmetric positive definite gives RN_ERR_INVAL. */
typedef struct {
  double W_alpha;
  const double *alpha0;
  const double *Wu;
  double Ws, Wx;
} rn_cost;

/* Options of the factor step.  Zero-initialise for the defaults. */
typedef struct {
  int device;          /* CUDA device ordinal */
  void *stream;        /* cudaStream_t for all work of this handle; NULL =
                          a stream owned by the handle */
  int precision;       /* rn_precision */
  double gamma;        /* APG step; 0 = 1 / (1.01 L) with L from power
                          iteration on the dual Hessian */
  int power_iters;     /* 0 = 200 */
  int check_every;     /* residual test every k iterations; 0 = 10 */
  int refresh_every;   /* RN_PREC_MIXED: FP64 reference refresh period;
                          0 = 40 (periods of 20 to 40 gave the same
                          distance from the FP64 iterate on the
                          512-scenario tree at 300 to 2,000 iterations;
                          each refresh costs one FP64 evaluation) */
  int max_ctas;        /* cap on the persistent grid; 0 = device maximum.
                          The handle's own kernels need one resident block
                          per work item (one per group of top nodes and per
                          set of chain teams, grid_ctas of
                          rapidnet_factor_info with max_ctas = 0): a smaller
                          cap gives RN_ERR_UNSUPPORTED at factor creation.
                          rapidnet_solve_batch takes the cap of its first
                          handle for the batch's grid, where a block may
                          take several work items. */
  int block_threads;   /* threads of a chain team of the persistent kernels
                          (multiple of 32, <= 256; a block is two or four
                          teams); 0 = one thread per component of u or x,
                          at least 64 */
  int wait_us;         /* bound of every device-side wait (a block waiting
                          for another block's flag or counter), in
                          microseconds; 0 = 2 s.  A wait that runs out ends
                          the launch with RN_ERR_TIMEOUT and the site of the
                          wait in rapidnet_last_error(); the handle stays
                          usable. */
  int theta_rule;      /* extrapolation sequence of the APG (paper §4.3,
                          which names two admissible choices):
                          RN_THETA_EQUALITY (0, default) theta_{nu+1} =
                          (sqrt(theta^4 + 4 theta^2) - theta^2) / 2, or
                          RN_THETA_SIMPLE theta_nu = 2 / (nu + 2); both from
                          theta_0 = theta_{-1} = 1 and beta_nu = theta_nu
                          (1 / theta_{nu-1} - 1) */
  int batch_tune;      /* rapidnet_solve_batch, read from the batch's first
                          handle: 0 (default) times the candidate launch
                          layouts (team width, teams per block) on a short
                          run of the first batch of a set of handles, keeps
                          the fastest for later batches of that set, and
                          replays the batch as a captured CUDA graph; 1 the
                          rule-based layout, as a graph; 2 the rule-based
                          layout launched directly (no graph) */
  int factor_form;     /* RN_FACTOR_AUTO (0), RN_FACTOR_SHARED or
                          RN_FACTOR_PER_NODE */
} rn_opts;

enum { RN_THETA_EQUALITY = 0, RN_THETA_SIMPLE = 1 };

/* Output of a solve.  The caller allocates u (n_nodes*nu), x (n_nodes*nx)
 * and y (n_nodes*(2 nx + nu)) in the memory space of the call (host for
 * rapidnet_solve, device for rapidnet_solve_device); res_hist (may be
 * NULL) receives one residual per check, at most res_hist_len.  Root
 * rows: u = q, x = x0, y = 0. */
typedef struct {
  double *u, *x, *y;
  double *res_hist;
  int res_hist_len;
  int compute_gap;     /* nonzero: also evaluate the duality gap (one more
                          dual-gradient evaluation) */
  /* filled by the call */
  int iters;           /* APG iterations performed */
  int n_checks;        /* residual checks performed */
  double primal_res;   /* |H x*(w) - t|_inf of the last iteration */
  double ubox_viol;    /* max violation of umin <= u <= umax by u* */
  double cost;         /* objective of eq. SMPC at (u*, x*) without the
                          indicator of the input box */
  double gap;          /* cost(x*(y)) - dual value at y (NaN unless
                          compute_gap) */
  double gamma;        /* step size used */
  double apg_ms;       /* device time of the APG iterations (CUDA events on
                          the handle's stream around the persistent launch) */
  long long t_begin_ns, t_end_ns;  /* device clock (%globaltimer, ns) when the
                          persistent launch began and when its first block
                          finished; comparable between launches on one
                          device (0 from rapidnet_solve_batch) */
  double *u_avg, *x_avg;  /* NULL, or caller-allocated like u and x: the
                          averaged primal iterate of paper §4.3, which the
                          paper credits with an O(1/nu^2) rate,
                          xbar^nu = (1 - theta_nu) xbar^{nu-1} + theta_nu
                          x*(w^nu) from xbar^0 = x*(w^0) (theta_0 = 1),
                          accumulated in FP64 over the iterations.  Give
                          both or neither; rapidnet_solve_batch refuses them
                          (RN_ERR_UNSUPPORTED). */
} rn_result;

typedef struct rn_factor rn_factor;

/* Sizes and derived quantities of a factor handle. */
typedef struct {
  int nx, nu, nd, ne, N, n_nodes;
  int n_chains;        /* leaves = scenarios */
  int n_top;           /* nodes whose subtree holds more than one leaf */
  int grid_ctas;       /* blocks of the FP64 persistent kernel */
  int block_threads;   /* threads per block (two chain teams) */
  double L;            /* power-iteration estimate of the dual Lipschitz
                          constant (0 if gamma was given) */
  double gamma;
  int precision;
  long long device_bytes;  /* device memory held by the handle */
  double collapse_dev;     /* factor check: max |2 p Phi - F| / max |F| over
                              the sampled nodes of the general recursion */
  long long noalloc_bytes; /* scratch that rapidnet_dual_gradient_noalloc
                              needs for this handle's tree (compare with
                              RN_NOALLOC_SCRATCH_BYTES) */
  int factor_form;         /* RN_FACTOR_SHARED or RN_FACTOR_PER_NODE */
} rn_factor_info;

/* Factor step (paper Table 2 Engine::factorStep, §4.4): validates the
 * inputs, builds the tree schedule, the Schur complement E W_u^-1 E' and
 * its inverse (FP64), uploads everything to the device, and, unless
 * opts->gamma > 0, estimates the Lipschitz constant of the dual gradient
 * by FP64 power iteration.  On success *out owns device memory until
 * rapidnet_factor_free.  opts may be NULL (defaults).
 * The factor check runs one step of the general per-node recursion
 * (Q = 2 p W_u + sum of the children's P, Phi = L (L' Q L)^-1 L', L a
 * basis of ker E) in FP64 at the first node of stages 1, N/2 and N, and
 * returns RN_ERR_RANK if 2 p Phi differs from the shared operator F by more
 * than 1e-8 relative (E W_u^-1 E' too ill-conditioned).  The shared form
 * returns RN_ERR_UNSUPPORTED, before any launch, for A != I,
 * nx or nu above 256, or a tree whose schedule needs more work items than
 * the device keeps resident (one item per group of top nodes and per four
 * chains), a group larger than the shared-memory capacity, or a dense W_u
 * with chain teams narrower than nu / 2 threads (block_threads); with
 * RN_FACTOR_AUTO and RN_PREC_FP64 such a refusal is followed by the
 * per-node form.
 * The per-node form (RN_FACTOR_PER_NODE; RN_FACTOR_AUTO for A != I or
 * RN_PREC_FP32) runs the general recursion at every node on the host in
 * FP64 (one worker thread per core), uploads Phi_nu and K_nu in the
 * iteration's precision (rows padded to 16 bytes: 2 nu^2 values per node,
 * 1.1 GB in FP32 for 10^4 nodes of nu = 114) and (I - Phi_nu Q_nu) E' in
 * FP64, and estimates L by power iteration in the iteration's precision
 * (FP64 with RN_PREC_MIXED).
 * With RN_PREC_MIXED it holds both an FP32 and an FP64 set (the FP64 one
 * evaluates x*(yb) at every refresh and the final primal).
 * It returns RN_ERR_INVAL where L' Q L is not positive definite at some
 * node, RN_ERR_UNSUPPORTED for nx or nu above 1024. */
int rapidnet_factor(const rn_network *net, const rn_tree *tree,
                    const rn_cost *cost, const rn_opts *opts,
                    rn_factor **out);

/* The per-node matrices of the general recursion (paper §4.4) as the
 * per-node form's factor step computes them, in FP64 on the host, with no
 * device work: Phi (n_nodes*nu*nu), K (n_nodes*nu*nu) and Mc (n_nodes*nu*ne,
 * may be NULL) = (I - Phi_nu Q_nu) E', row-major per node, root rows zero.
 * Caller-allocated host arrays.  RN_OK, RN_ERR_INVAL, RN_ERR_RANK. */
int rapidnet_pernode_matrices(const rn_network *net, const rn_tree *tree,
                              const rn_cost *cost, double *Phi, double *K,
                              double *Mc);
void rapidnet_factor_free(rn_factor *f);
int rapidnet_factor_info(const rn_factor *f, rn_factor_info *info);

/* One solve (paper Table 2 SmpcController::controlAction): APG from
 * y_warm (NULL = 0; n_nodes*(2nx+nu), also used as y^{-1}) for at most
 * max_iters iterations, stopping at the first check with residual <= tol
 * (tol <= 0: run exactly max_iters).  Host pointers: x0 (nx), q (nu),
 * demand (n_nodes*nd, row 0 ignored), alpha (n_nodes*nu, row 0 ignored).
 * Copies in and out on the handle's stream and synchronises it.
 * Returns RN_OK (converged), RN_NOT_CONVERGED, or an error. */
int rapidnet_solve(rn_factor *f, const double *x0, const double *q,
                   const double *demand, const double *alpha, int max_iters,
                   double tol, const double *y_warm, rn_result *out);

/* Same as rapidnet_solve with every array argument (inputs, y_warm, and
 * out->u, x, y, res_hist) a DEVICE pointer on the handle's device.
 * Synchronises the handle's stream before returning (the scalars of *out
 * are read back). */
int rapidnet_solve_device(rn_factor *f, const double *x0, const double *q,
                          const double *demand, const double *alpha,
                          int max_iters, double tol, const double *y_warm,
                          rn_result *out);

/* One problem of a batch: device pointers as for rapidnet_solve_device;
 * out->u, x, y (device) receive the outputs and out's scalars are filled. */
typedef struct {
  const double *x0, *q, *demand, *alpha;
  const double *y_warm;  /* NULL = cold start */
  rn_result *out;
} rn_solve_req;

/* Batched solve: n independent problems, each on its own factor handle
 * (different networks and trees allowed, all created with
 * RN_PREC_MIXED on one device), run together in one persistent
 * cooperative launch on the stream of f[0] (the paper solves one problem
 * at a time; this serves many MPC problems at once).  Every problem runs
 * at most max_iters iterations and
 * stops at its own first check with residual <= tol (tol <= 0: exactly
 * max_iters).  Returns RN_OK when every problem converged (or tol <= 0),
 * RN_NOT_CONVERGED when some did not, or an error; per-problem results in
 * req[i].out.  Synchronises the streams of all handles.  RN_ERR_UNSUPPORTED
 * (before any launch) when a problem's group of top nodes does not fit the
 * batch's shared-memory layout, when a handle has a dense W_u (the batched
 * kernel applies F in its sparse form only) or when a request asks for the
 * averaged primal iterate.  A call runs every problem's preparation, the
 * batched kernel and the outputs on the stream of f[0] (the other handles'
 * streams are synchronised first), with one read-back of all problems'
 * scalars; the library keeps the last batch's work space and CUDA graph per
 * device and replays the graph when the next call has the same handles,
 * requests, max_iters and tol.  out->apg_ms is the device time of the whole
 * sequence (preparations, batched kernel, outputs);
 * t_begin_ns and t_end_ns are 0. */
int rapidnet_solve_batch(rn_factor *const *f, const rn_solve_req *req, int n,
                         int max_iters, double tol);

/* Dual gradient x*(w) = grad f*(-H'w) (eq. dual-gradient, §4.4) for the
 * data of the last solve, or of (x0, q, demand, alpha) when given (all
 * device pointers, NULL = keep the last solve's data): w (n_nodes*(2nx+nu),
 * row 0 ignored) in, u (n_nodes*nu) and x (n_nodes*nx) out, device
 * pointers, FP64.  Synchronises the handle's stream. */
int rapidnet_dual_gradient_device(rn_factor *f, const double *x0,
                                  const double *q, const double *demand,
                                  const double *alpha, const double *w,
                                  double *u, double *x);

/* Dual gradient without allocation.  The paper has no counterpart: this
 * serves callers that must not allocate device memory after start-up (a
 * real-time control loop with a no-allocation rule for predictable
 * timing, or a host that owns the device memory pool).  Such a caller
 * creates the handle and runs one solve (or rapidnet_dual_gradient_device
 * with data) during set-up; this call then gives the same result as
 * rapidnet_dual_gradient_device for the data of that last solve: w in
 * (n_nodes*(2nx+nu)), u (n_nodes*nu) and x (n_nodes*nx) out, all device
 * pointers, FP64.
 * Scratch: one fixed array of RN_NOALLOC_SCRATCH_BYTES (8 MiB) of device
 * memory inside the library, held by every device that loads the library
 * until the process exits.  A tree needs
 *   8 (n (3 sp + 2 nup + nxp) + 2 max(h, 1) sp) + 4 (3 max(g, 1) + 6)
 * bytes (rounded up to 8), with n = n_nodes, nxp / nup = nx / nu rounded
 * up to multiples of 4, sp = nxp + nup, h the rows of partial sums of
 * split stage-1 subtrees and g the groups plus roots of the schedule
 * (h, g < n); rapidnet_factor_info's noalloc_bytes gives the exact figure.
 * Larger trees get RN_ERR_INVAL.  The Barcelona-sized network needs 836
 * doubles per node, so about 1,250 nodes fit: its 32-scenario tree (701
 * nodes) does, its 512-scenario tree does not.
 * No cudaMalloc, cudaFree or allocating routine is called.  The first
 * call on a device looks up the array's device address
 * (cudaGetSymbolAddress); make that first call before any stream capture.
 * Every call shares the one array and finds the previous call's contents
 * in it: calls that overlap on the GPU (other streams, handles or host
 * threads) race and must be serialised by the caller.  Copies the error
 * word back and synchronises the handle's stream before returning. */
#define RN_NOALLOC_SCRATCH_BYTES (8LL << 20)
int rapidnet_dual_gradient_noalloc(rn_factor *f, const double *w, double *u,
                                   double *x);

/* ---------------------------------------------------------------------
 * Serving: continuous batching of solve requests (no counterpart in the
 * paper, which solves one problem per control step).  A server holds
 * models (network x tree x cost), each served by one or more slots: a
 * resident factor handle with its own stream, device buffers and the last
 * dual it computed (warm start).  Submitted requests wait in a bounded
 * queue; worker threads take a request as soon as its model has a free
 * slot, or open a new slot when the device-memory budget allows, and run
 * it on that slot's stream, so requests that arrive while others run
 * overlap with them on the device.  Every result equals the same request
 * solved alone (same kernels, no shared state besides the warm start,
 * which is off unless asked for).  A model takes its factor form as
 * rapidnet_factor does (RN_FACTOR_AUTO: the shared form where it applies);
 * solves of per-node models fill the device and run one at a time.
 * ------------------------------------------------------------------- */
typedef struct rn_server rn_server;

typedef struct {
  int device;
  long long budget_bytes;  /* device memory the slots may hold; 0 = 8 GiB */
  int max_queue;           /* pending requests; 0 = 4096 */
  int workers;             /* concurrent solves (host threads); 0 = 8 */
  int slots_per_model;     /* slots opened when a model is added (within the
                              budget); 0 = 1.  Later slots are opened on
                              demand; opening one allocates device memory,
                              which briefly stalls the device */
} rn_server_opts;

typedef struct {
  long long submitted, completed, rejected;
  int slots, models;
  long long bytes_in_use;
  double p50_s, p99_s;     /* latency (submit -> result ready) of completed */
  double mean_s;
} rn_server_stats;

int rapidnet_server_create(const rn_server_opts *opts, rn_server **out);
/* Adds a model; its first slot (a factor handle) is created now and
 * charged to the budget.  opts as for rapidnet_factor (device taken from
 * the server).  *key identifies the model in submit. */
int rapidnet_server_add_model(rn_server *s, const rn_network *net, const rn_tree *tree,
                              const rn_cost *cost, const rn_opts *opts, int *key);
/* Queues one solve; host arrays are copied.  warm != 0 starts from the
 * last dual of the slot that runs it.  Returns RN_ERR_NOMEM when the queue
 * is full (retry later), RN_ERR_INVAL for a bad key. */
int rapidnet_server_submit(rn_server *s, int key, const double *x0, const double *q,
                           const double *demand, const double *alpha, int max_iters,
                           double tol, int warm, long long *ticket);
/* Waits up to timeout_s (< 0: no limit) for a ticket; fills out (host
 * buffers u, x, y may be NULL) and the latency.  Returns the solve's
 * status, or RN_ERR_TIMEOUT if it is not done yet.  A ticket is returned
 * once; later calls give RN_ERR_INVAL. */
int rapidnet_server_wait(rn_server *s, long long ticket, double timeout_s, rn_result *out,
                         double *latency_s);
int rapidnet_server_stats(rn_server *s, rn_server_stats *st);
/* Finishes the queued requests, then frees every slot. */
void rapidnet_server_destroy(rn_server *s);

/* ---------------------------------------------------------------------
 * Scenario tree from sampled paths (paper §2.3 and §6.2: Monte-Carlo
 * scenarios reduced into a tree; the paper cites Heitsch and Römisch).
 * The tree is built forward: every node of stage t holds a bundle of the
 * paths (the root all of them); its min(branching[t], bundle size)
 * children are representatives chosen by fast forward selection on the
 * distance between the paths' remaining parts (stages t+1 .. N,
 * Euclidean over stages and dimensions), one at a time, each minimising
 * sum_j p_j min(m_j, d(j, u)) with m_j the distance of path j to the
 * nearest representative chosen so far (lowest index on ties); every path
 * goes to its nearest representative (first chosen on ties).  A child
 * carries its representative's value at its stage and the probability of
 * its paths.  Distances, selection and assignment run on the GPU in FP64.
 * ------------------------------------------------------------------- */
typedef struct {
  int max_nodes;     /* capacity of anc, prob, rep (and value / dim) */
  int n_nodes;       /* filled: nodes of the tree, breadth first */
  int *stage_ptr;    /* N + 2: nodes of stage t are [stage_ptr[t], stage_ptr[t+1]) */
  int *anc;          /* ancestor of each node, anc[0] = -1 */
  double *prob;      /* probability of reaching each node */
  double *value;     /* n_nodes * dim: the node's value (row 0 zero) */
  int *rep;          /* the path each node represents (-1 at the root) */
  int *leaf_of;      /* S: the leaf of every path */
} rn_tree_out;

/* paths: host, S * N * dim row-major (path s, stage t + 1, component);
 * prob: S, adding up to 1 (NULL: uniform); branching: N entries >= 1.
 * Output arrays are host memory allocated by the caller.  Returns RN_OK,
 * RN_ERR_INVAL (bad sizes, probabilities, non-finite values, or more nodes
 * than max_nodes), RN_ERR_NOMEM or RN_ERR_CUDA.  Work space on the device:
 * S * S doubles for the distance matrix plus O(S * N * dim). */
int rapidnet_scenario_tree(const double *paths, const double *prob, int S, int N, int dim,
                           const int *branching, int device, rn_tree_out *out);

/* Description of the last failure on the calling thread ("" if none). */
const char *rapidnet_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* RAPIDNET_H */
