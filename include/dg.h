/*
 * dg.h -- C ABI of libdg: the GB300 (sm_103a) DGSEM residual, Williamson RK3
 * step and unsteady anisotropic tau-estimation sweep of Rueda-Ramirez,
 * Ntoukas, Rubio, Valero, Ferrer, "Truncation Error-Based Anisotropic
 * p-Adaptation for Unsteady Flows for High-Order Discontinuous Galerkin
 * Methods" (arXiv 2210.03523).
 *
 * Conventions shared by every entry point
 * ---------------------------------------
 * Element e has orders (N1,N2,N3), 1 <= N_i <= DG_MAX_ORDER, and
 * n_e = (N1+1)(N2+1)(N3+1) Gauss-Lobatto (GL) nodes.  A "state-layout"
 * array holds 5 doubles per node: element e starts at 5*off_e, off_e =
 * sum_{e'<e} n_e', and is ordered [var][k][j][i] (i fastest) with
 * var = (rho, rho u, rho v, rho w, rho E).  Faces of an element are numbered
 * 0..5 = (-xi1, +xi1, -xi2, +xi2, -xi3, +xi3).
 *
 * Memory: every pointer called "device" is CUDA device memory of the
 * current device, owned and allocated by the caller; "host" pointers are
 * read during the call only.  The mesh owns its geometry, connectivity and
 * scratch buffers.  Calls are asynchronous on the mesh's CUDA stream unless
 * stated otherwise.  Argument errors are returned synchronously and leave
 * the device untouched.  Device-side errors (a non-physical state: rho <= 0,
 * p <= 0 or NaN) set a sticky error word that dg_get_error() returns.
 * A mesh is not thread-safe.
 */
#ifndef DG_H
#define DG_H

#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

#define DG_MAX_ORDER 8

typedef enum {
  DG_OK = 0,
  DG_ERR_ARG = 1,          /* invalid argument (null pointer, order out of range, bad connectivity) */
  DG_ERR_NOMEM = 2,        /* device or host allocation failed */
  DG_ERR_CUDA = 3,         /* a CUDA runtime call failed */
  DG_ERR_UNSUPPORTED = 4,  /* valid input outside what the library implements */
  DG_ERR_NONPHYSICAL = 5,  /* sticky device error: rho <= 0, p <= 0 or NaN met */
  DG_ERR_TIMEOUT = 6,      /* reserved: a bounded device wait gave up */
  DG_ERR_INDEX = 7         /* sticky device error of the bounds-checking build: a kernel met an index out of
                              range in a work list and skipped that unit of work */
} dg_status;

enum { DG_EULER = 0, DG_NAVIER_STOKES = 1 };

/* boundary tags in dg_mesh_desc.neighbors */
enum { DG_BC_FARFIELD = -1, DG_BC_WALL = -2 };

/* dg_residual flags */
#define DG_ISOLATED 0x1u        /* isolated residual: inner flux on every face (Sec. 2.2, end) */

/* dg_tau_estimate flags */
#define DG_TAU_ISOLATED 0x1u    /* isolated tau (the paper's results use it, Sec. 3); else non-isolated */
#define DG_TAU_FP32 0x2u        /* sweep arithmetic and maps in float; else double */
#define DG_TAU_ACCUM_MAX 0x4u   /* map = max(map, new): F_max over estimation stages (Sec. 2.4) */

/* Gas model (Sec. 2.1, Eq. NScons/SystemAdvDiff): ideal gas with ratio of
 * specific heats gamma and gas constant Rgas (T = p/(rho Rgas)); for
 * Navier-Stokes a constant viscosity mu, Stokes hypothesis and Fourier heat
 * flux with kappa = mu gamma Rgas / ((gamma-1) Pr).  q_inf is the
 * free-stream conservative state used by DG_BC_FARFIELD. */
typedef struct {
  int32_t eqs;       /* DG_EULER or DG_NAVIER_STOKES */
  double gamma, mu, Pr, Rgas;
  double q_inf[5];
} dg_physics;

/* Mesh description (all host memory, copied by dg_mesh_create).
 * geom: [n_elem][(G+1)^3][3] node coordinates of each element's degree-G
 *       geometry on the equispaced reference lattice xi = -1 + 2a/G,
 *       index a + (G+1)(b + (G+1)c); the element map is the degree-G
 *       tensor polynomial through them (Sec. 2.1: J_j of the geometry
 *       transformation).
 * neighbors: [n_elem][6]; >= 0: the element across that face, whose
 *       opposite face (f^1) must point back, with aligned reference axes;
 *       < 0: a DG_BC_* tag.
 * orders: [n_elem][3] per-direction orders (Sec. 2.4: p-anisotropic). */
typedef struct {
  int32_t n_elem;
  int32_t geom_order;
  const double* geom;
  const int32_t* neighbors;
  const int32_t* orders;
  dg_physics phys;
} dg_mesh_desc;

typedef struct dg_mesh dg_mesh;

/* Builds geometry, Kopriva curl-form metric terms, face connectivity and
 * (N1,N2,N3) buckets, and uploads them.  stream: a cudaStream_t, or NULL
 * for the legacy default stream.  Synchronous.
 * Mortars (p-nonconforming faces) of order max(N_L, N_R) per tangential
 * direction: on affine Euler meshes one Roe flux per mortar node serves both
 * sides; on curved or Navier-Stokes meshes each side takes the flux with its
 * own J a^dir interpolated to the mortar (the two elements' metrics differ
 * at a curved nonconforming face), with the BR1 averages of q and of the
 * viscous flux formed on the mortar.
 * Errors: DG_ERR_ARG (null pointer, order outside 1..DG_MAX_ORDER,
 * neighbour index out of range or not reciprocal, unknown tag, J <= 0),
 * DG_ERR_NOMEM, DG_ERR_CUDA. */
dg_status dg_mesh_create(const dg_mesh_desc* desc, void* stream, dg_mesh** out);
/* Synchronises the mesh stream and frees everything the mesh owns (its
 * cached coarse meshes and CUDA graphs included).  Errors: DG_ERR_ARG (null). */
dg_status dg_mesh_destroy(dg_mesh* mesh);
/* Number of nodes and elements (host outputs; either may be NULL).
 * Errors: DG_ERR_ARG (null mesh). */
dg_status dg_mesh_info(const dg_mesh* mesh, int64_t* n_nodes, int32_t* n_elem);
/* The state layout (Sec. 2.1: the solution of element e holds its 5
 * variables at its (N1+1)(N2+1)(N3+1) GL nodes): *n_nodes the node count,
 * *elem_offset the device array off[0..n_elem] (int64) with element e's
 * nodes at off[e] .. off[e+1]-1, so its values start at 5 off[e] in a state
 * array, [var][k][j][i] with i fastest.  The array is owned by the mesh and
 * valid until dg_set_orders or dg_mesh_destroy; either output may be NULL.
 * Errors: DG_ERR_ARG (null mesh). */
dg_status dg_mesh_layout(const dg_mesh* mesh, int64_t* n_nodes, const int64_t** elem_offset);
/* Number of nodes sum_e prod_i (N_i+1) of a layout with the given host
 * orders [n_elem][3]; host only.  Errors: DG_ERR_ARG (n_elem < 0, null
 * orders with n_elem > 0, null n_nodes, an order outside 1..DG_MAX_ORDER). */
dg_status dg_count_nodes(int32_t n_elem, const int32_t* orders, int64_t* n_nodes);
/* Later calls on the mesh (and its cached coarse meshes) run on stream (a
 * cudaStream_t, or NULL for the legacy default stream); ordering against
 * work already queued on the previous stream is the caller's.
 * Errors: DG_ERR_ARG (null mesh). */
dg_status dg_set_stream(dg_mesh* mesh, void* stream);

/* Node coordinates: device xyz[3*n_nodes], element e at 3*off_e as
 * [d][node].  Synchronous.  Errors: DG_ERR_ARG (null pointer), DG_ERR_CUDA. */
dg_status dg_node_coords(dg_mesh* mesh, double* xyz);

/* Residual R(Q) = dQ/dt = -(M^N)^{-1} F^N(Q) of the DGSEM discretisation,
 * Sec. 2.1, Eqs. (DGSEMsystem), (DGMassMatrixLeft), (DGMassMatrixRight):
 * Roe advective flux and, for Navier-Stokes, BR1 for q-hat and the viscous
 * flux (Sec. 3); p-nonconforming faces through mortars of order
 * max(N_L, N_R) per tangential direction.  flags: DG_ISOLATED gives the
 * isolated residual (surface numerical fluxes replaced by the inner flux,
 * end of Sec. 2.2).  q, r: device, state layout, FP64; r may not alias q.
 * Errors: DG_ERR_ARG, DG_ERR_UNSUPPORTED (a mortar batch above the device's
 * shared memory, which no order up to DG_MAX_ORDER reaches), DG_ERR_CUDA. */
dg_status dg_residual(dg_mesh* mesh, const double* q, double* r, uint32_t flags);

/* Residual without any device allocation.  The paper has no counterpart:
 * this entry point exists for callers that may not call cudaMalloc while
 * they run, for instance code inside a framework whose pooling allocator
 * already owns the device memory budget (a raw cudaMalloc there can fail or
 * fragment the pool), or a loop that must not stall on the device-wide
 * synchronisation that cudaMalloc / cudaFree may imply.
 * It returns the same R(Q) as dg_residual(mesh, q, r, 0) for Euler meshes,
 * but its face-flux scratch is one fixed array inside the library
 * (DG_NOALLOC_SURF_DOUBLES = 4,194,304 doubles, 32 MiB, reserved on every
 * GPU that loads the library until the process exits) instead of the
 * mesh's buffer.  It calls no cudaMalloc, cudaFree or allocating library
 * routine.
 *   q, r: device state-layout arrays as for dg_residual; r may not alias q.
 *   The mesh's device must be the current device.
 *   Each call looks up the array's device address on the current device
 *   (cudaGetSymbolAddress), so the address always belongs to the live
 *   context, also after a cudaDeviceReset.  While the mesh stream is being
 *   captured the address of the last lookup on that device is used instead:
 *   make one call on the device before any stream capture (a first call
 *   during capture returns DG_ERR_CUDA).  Several host threads may call at
 *   the same time.
 *   All calls share the one array: calls that overlap on the GPU (two
 *   streams, two meshes) race on it and must be serialised by the caller.
 *   Every call rewrites the whole part of the array it reads, so nothing
 *   carries over from an earlier call.
 * Errors: DG_ERR_ARG (null or aliased pointers, mesh device not current),
 * DG_ERR_UNSUPPORTED (Navier-Stokes mesh, a mortar batch above the device's
 * shared memory as for dg_residual, or a face buffer of more than
 * DG_NOALLOC_SURF_DOUBLES doubles: 5 per element-face node, i.e. more than
 * 838,860 element-face nodes), DG_ERR_CUDA. */
#define DG_NOALLOC_SURF_DOUBLES 4194304
dg_status dg_residual_noalloc(dg_mesh* mesh, const double* q, double* r);

/* CFL time step (Sec. 3: dt adapted from the CFL condition each step):
 * dt = cfl / max_nodes max(s_a, s_v),
 *   s_a = sum_i (N_i+1)^2 (|J a^i . v| + c |J a^i|) / (2J),
 *   s_v = sum_i (N_i+1)^4 |J a^i|^2/(4J^2) max(1, gamma/Pr) mu/rho (NS only).
 * q: device state; dt_dev: device double written on the stream, so that a
 * captured RK loop can consume it without a host round trip.
 * Errors: DG_ERR_ARG (null pointer, cfl not > 0), DG_ERR_CUDA; a
 * non-physical state sets the sticky error word. */
dg_status dg_max_dt(dg_mesh* mesh, const double* q, double cfl, double* dt_dev);

/* One step of Williamson's low-storage RK3 (Sec. 3), stages k = 1..3:
 *   G <- A_k G + dt R(Q),  Q <- Q + B_k G,
 * A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15).  q and g (the RK
 * register, zero before the first step) are device state-layout arrays
 * updated in place; dt_dev is a device double read by the kernels.
 * Errors: DG_ERR_ARG (null pointer, q == g), DG_ERR_UNSUPPORTED (as
 * dg_residual), DG_ERR_CUDA; a non-physical state sets the sticky error
 * word. */
dg_status dg_rk_step(dg_mesh* mesh, double* q, double* g, const double* dt_dev);

/* Unsteady anisotropic tau-estimation, variational DG form (Sec. 2.3 item 1):
 *   new form (Eq. TEtildedef):  tau~^N = I_{N<-P} R^P(q^P) - R^N(I_{N<-P} q^P)
 *   traditional (Eq. TEdef):    tau^N  = M^N tau~^N = J_j w_j tau~^N_j
 * with I_{N<-P} interpolation from the element's orders P to N, for every
 * element e and every sweep entry s (orders N_s).  The map entry is the
 * infinity norm over the element's nodes and all five variables if
 * N_s <= P_e componentwise, else -1.
 *   q: device state (q^P); r_p: device state R^P or NULL (then R^P is the
 *      residual of the same variant as R^N, so tau at N = P is exactly 0).
 *      The full residual of the time stepper gives the literal variational
 *      form; the physical time derivative delta_p/delta_t q^P of a dual
 *      time-stepping integrator gives the dual time-stepping estimate
 *      (Sec. 2.3 item 2): the time discretisation is linear, so
 *      delta_p/delta_t (I q^P) = I (delta_p/delta_t q^P);
 *   sweep: host [n_sweep][3]; map_new / map_trad: device [n_elem][n_sweep],
 *      float if DG_TAU_FP32 else double; either may be NULL (not written).
 *   flags: DG_TAU_ISOLATED (element-local residuals; coarse geometry is the
 *      element map interpolated to N), else non-isolated (full residual of
 *      the coarse discretisation with orders min(N_s, P_e) in every
 *      element); DG_TAU_FP32; DG_TAU_ACCUM_MAX.
 * Asynchronous on the mesh stream.  Errors: DG_ERR_ARG (null q or sweep,
 * n_sweep <= 0, both maps NULL, unknown flag bits, an order outside
 * 1..DG_MAX_ORDER); DG_ERR_UNSUPPORTED (isolated: a tile class whose sweep
 * needs more shared memory than the device offers, as FP64 does for
 * elements of 9 x 9 x 9 nodes, where DG_TAU_FP32 serves; non-isolated: as
 * dg_residual); DG_ERR_NOMEM; DG_ERR_CUDA. */
dg_status dg_tau_estimate(dg_mesh* mesh, const double* q, const double* r_p, const int32_t* sweep, int32_t n_sweep,
                          uint32_t flags, void* map_new, void* map_trad);

/* Work units of the isolated sweep (DG_TAU_ISOLATED).  Sec. 2.3 estimates
 * tau at every coarser N of every element; the library runs a tile of
 * same-order elements and some of its sweep entries as one unit of work.
 * Sweep entries sharing (N2, N3) form a group; a unit holds either one
 * group, or every group of one N3 (the xi3 restriction of q^P and R^P is
 * then computed once for all of them).  How entries are split into units
 * changes no node's arithmetic: the maps are bitwise the same in every mode.
 *   mode DG_TAU_UNITS_AUTO (default): groups shared, except in a shared-
 *        memory size class that would have fewer than 8 x 152 units (too few
 *        CTAs to fill the GPU), where each unit holds one group;
 *   DG_TAU_UNITS_GROUPED: groups shared in every class;
 *   DG_TAU_UNITS_SPLIT: one group per unit in every class.
 * The mode takes effect at the next isolated dg_tau_estimate (the units are
 * rebuilt on the host then, synchronously) and survives dg_set_orders.
 * Errors: DG_ERR_ARG (null mesh, unknown mode). */
#define DG_TAU_UNITS_AUTO 0
#define DG_TAU_UNITS_GROUPED 1
#define DG_TAU_UNITS_SPLIT 2
dg_status dg_set_tau_units(dg_mesh* mesh, int32_t mode);
/* The units of the last isolated sweep's list, per shared-memory size class
 * (host outputs): *n_classes the number of classes (0 before the first
 * isolated sweep, or after dg_set_tau_units); for k < min(*n_classes,
 * max_classes), n_units[k] the units and n_shared[k] those holding two or
 * more groups.  Errors: DG_ERR_ARG (null mesh or n_classes, max_classes < 0,
 * null arrays with max_classes > 0). */
dg_status dg_tau_units_info(const dg_mesh* mesh, int32_t max_classes, int32_t* n_classes, int32_t* n_units,
                            int32_t* n_shared);

/* Change the element orders to new_orders (host [n_elem][3]) and project
 * the state (Sec. 2.4: after adaptation the storage is reallocated and the
 * solution projected to the new polynomial spaces): per direction,
 * interpolation when the order rises and L2 projection when it falls.
 * q_old: device, old layout; q_new: device, new layout of
 * dg_count_nodes(new_orders) nodes, caller-allocated, not aliasing q_old.
 * The mesh is rebuilt for the new orders (synchronous); on an error it is
 * left as it was.  Errors: DG_ERR_ARG (null pointer, q_old == q_new, an
 * order outside 1..DG_MAX_ORDER), DG_ERR_NOMEM, DG_ERR_CUDA. */
dg_status dg_set_orders(dg_mesh* mesh, const int32_t* new_orders, const double* q_old, double* q_new);

/* p-adaptation, order selection (Sec. 2.4, approach 2; with the degree-jump
 * conditions of Sec. 3.1, Eqs. N23 and N_1).  From a total truncation-error
 * map (a dg_tau_estimate map, F_max-accumulated over the estimation stages
 * of the static strategy, or a dg_tau_extrapolate map over a target list),
 * for every element: the sweep entry N with 0 <= map < tau_max and
 * n_min <= N_i <= n_max of fewest degrees of freedom prod_i (N_i+1), the
 * first in sweep order on ties; n_max in every direction when no entry
 * qualifies (entries above the element's own orders are -1 and never
 * qualify).  max_decrease >= 0 (dynamic adaptation, Sec. 3.3: the orders
 * fall by at most one per stage) raises each order to at least the mesh's
 * current order minus max_decrease (capped at n_max); < 0: no limit.  Then
 * the jump condition, as the least orders at or above that selection that
 * satisfy it: jump_rule 1: N_i^e >= floor(2 N_i^j / 3); 2: N_i^e >=
 * N_i^j - 1 for every face neighbour j; 0: none.  map: device
 * [n_elem][n_sweep], float if map_fp32 else double; sweep: host, the list
 * the map was built over; orders_out: host [n_elem][3], ready for
 * dg_set_orders.  Synchronous.
 * Errors: DG_ERR_ARG (null pointers, tau_max <= 0, bad bounds or rule). */
dg_status dg_select_orders(dg_mesh* mesh, const void* map, int32_t map_fp32, const int32_t* sweep, int32_t n_sweep,
                           double tau_max, int32_t n_min, int32_t n_max, int32_t jump_rule, int32_t max_decrease,
                           int32_t* orders_out);

/* Truncation-error extrapolation to N_i >= P_i (Sec. 2.3; Sec. 2.4:
 * approach 2 needs the extrapolated map of every estimation stage, and a
 * direction that cannot be extrapolated gets a high value).  For every
 * element with orders P and its map over the sweep (a dg_tau_estimate map):
 *   d_i(n): the map at the orders P with N_i = n < P_i (the directional
 *     entries present in the sweep);
 *   fit: the least-squares line through (n, ln d_i(n)) over the last n_fit
 *     points below P_i (all when n_fit <= 0), positive values only; with at
 *     least two points and a negative slope, e_i(n) = exp(a_i + b_i n);
 *     if d_i(P_i - 1) <= tau_floor the direction is resolved, e_i = 0;
 *     otherwise e_i = +infinity (P_i <= 2 always ends here);
 *   value at a target N: coupled (default): map(min(N, P)) + sum over
 *     N_i >= P_i of e_i(N_i), with map(P) = 0 and -1 when min(N, P) is not
 *     in the sweep; DG_EXTRAP_DECOUPLED: sum_i c_i(N_i), c_i(n) = d_i(n)
 *     below P_i and e_i(n) from P_i on (-1 when a needed d_i is missing),
 *     which needs only the sum_i (P_i - 1) directional sweep entries.
 * map: device [n_elem][n_sweep], float if map_fp32 else double; sweep:
 * host [n_sweep][3]; targets: host [n_targets][3], n_targets <= 512;
 * map_out: device [n_elem][n_targets] of the map's type; DG_EXTRAP_ACCUM_MAX
 * accumulates map_out = max(map_out, value) (F_max over stages).
 * Arithmetic in double.  Errors: DG_ERR_ARG. */
#define DG_EXTRAP_DECOUPLED 0x1u
#define DG_EXTRAP_ACCUM_MAX 0x2u
dg_status dg_tau_extrapolate(dg_mesh* mesh, const void* map, int32_t map_fp32, const int32_t* sweep, int32_t n_sweep,
                             const int32_t* targets, int32_t n_targets, int32_t n_fit, double tau_floor, uint32_t flags,
                             void* map_out);

/* Time integration to a given time (Sec. 3.1: the time step follows the
 * CFL condition at every step): Williamson RK3 steps of
 *   dt = min(cfl / max_nodes max(s_a, s_v), t_end - t)     (dg_max_dt's scale)
 * from the device time *t_dev; the step that reaches t_end sets *t_dev =
 * t_end exactly, and steps after it are empty (dt = 0 leaves q unchanged:
 * the first stage discards g).  At most max_steps steps.
 * t_end = +infinity: exactly max_steps CFL steps, asynchronous on the mesh
 * stream.  Otherwise the call returns once *t_dev = t_end or max_steps steps
 * were taken, reading the time back between batches of steps.
 * Steps run in batches captured once as CUDA graphs (on a private stream,
 * replayed on the mesh stream) and cached per (q, g, t_dev, batch size);
 * DG_ADVANCE_EAGER, or enabled profiling, launches them one by one instead.
 * q, g: device state and RK register as for dg_rk_step; t_dev: device
 * double; steps_out (host, optional): steps with dt > 0 in this call (a
 * synchronising read).  The cached graphs hold the buffers' addresses: free
 * q, g or t_dev only after the mesh, or pass other buffers (new graphs).
 * Errors: DG_ERR_ARG, DG_ERR_UNSUPPORTED (as dg_rk_step), DG_ERR_CUDA. */
#define DG_ADVANCE_EAGER 0x1u
dg_status dg_advance(dg_mesh* mesh, double* q, double* g, double* t_dev, double t_end, double cfl, int64_t max_steps,
                     uint32_t flags, int64_t* steps_out);

/* One pass of the hot path on host buffers: time stepping (Sec. 3.1) then
 * the estimate (Sec. 2.3) of one estimation stage.  The state q_in (host,
 * 5 * n_nodes doubles, state layout) is copied to the device, advanced by
 * dg_advance(t_end, cfl, max_steps) from time t0 with a zeroed RK register,
 * the sweep of dg_tau_estimate(tau_flags) is run on the advanced state, and
 * the state and the maps are copied back:
 *   q_out: host, 5 * n_nodes doubles (may equal q_in);
 *   map_new / map_trad: host [n_elem][n_sweep], float if DG_TAU_FP32 else
 *      double; either may be NULL (not computed), not both;
 *   t_out: host, optional: the time reached.
 * The device buffers are the mesh's own: allocated at the first call (and
 * again when the map size changes), kept until the mesh is destroyed or its
 * orders change; with DG_TAU_ACCUM_MAX the mesh's device maps keep the
 * F_max accumulation across calls (they start at 0).  Page-locked host
 * buffers make the copies asynchronous DMA on the mesh stream.  Synchronous:
 * returns once the copies back have finished.
 * The mesh's device must be the current device.
 * Errors: DG_ERR_ARG (null q_in, q_out or sweep, n_sweep <= 0, both maps
 * NULL, another device current), DG_ERR_NOMEM, then as dg_advance and
 * dg_tau_estimate. */
dg_status dg_step_host(dg_mesh* mesh, const double* q_in, double* q_out, double t0, double t_end, double cfl,
                       int64_t max_steps, const int32_t* sweep, int32_t n_sweep, uint32_t tau_flags, void* map_new,
                       void* map_trad, double* t_out);

/* Tile shapes (Sec. 2.4: elements of mixed anisotropic orders run in one
 * launch, bucketed by (N1,N2,N3)).  The volume kernels run one CTA per tile
 * of same-order elements, at most vol_budget nodes per tile (one element at
 * least) for the element-size class of the bucket: elements of <= 27, 125,
 * 343 or more nodes.  The mortar kernel runs one CTA per batch of same-shape
 * faces, at most mortar_budget mortar nodes per batch for the mortar-size
 * class: <= 9, 25, 49 or more mortar nodes.  Tiling does not change any
 * node's arithmetic: results are bitwise the same for every budget. */
#define DG_SIZE_CLASSES 4
#define DG_MAX_VOL_BUDGET 1024     /* 20 doubles of shared memory per node: 160 KB */
#define DG_MAX_MORTAR_BUDGET 512   /* up to 30 doubles per mortar node: 120 KB */
typedef struct {
  int32_t vol_budget[DG_SIZE_CLASSES];
  int32_t mortar_budget[DG_SIZE_CLASSES];
  double vol_ms[DG_SIZE_CLASSES];             /* dg_autotune: launch time after class k was tuned (-1: empty) */
  double vol_ms_default[DG_SIZE_CLASSES];     /* ... before */
  double mortar_ms[DG_SIZE_CLASSES];
  double mortar_ms_default[DG_SIZE_CLASSES];
} dg_tiles;

/* Autotuner of the tile shapes, by coordinate descent: for every size class
 * in turn (volume tiles first, then mortar batches), each candidate budget
 * (64, 128, 192, 256, 384, 512 nodes) with the other classes held is timed on
 * the whole production launch (the volume residual, or the face fluxes) on
 * this mesh and state: CUDA events on the mesh stream, the median of reps
 * launches after one warm-up.  The fastest is kept and the work lists are
 * rebuilt.  q: a device state of the mesh (physical, as for dg_residual);
 * out (host, optional): the chosen budgets; vol_ms[k] / mortar_ms[k] the
 * launch time after class k was tuned, *_default[k] before (-1: class
 * empty).  Synchronous.  Cached dg_advance graphs are released.
 * Errors: DG_ERR_ARG, DG_ERR_UNSUPPORTED (as dg_residual), DG_ERR_NOMEM,
 * DG_ERR_CUDA. */
dg_status dg_autotune(dg_mesh* mesh, const double* q, int32_t reps, dg_tiles* out);
/* The budgets in use (times -1).  Errors: DG_ERR_ARG (null pointer). */
dg_status dg_get_tiles(const dg_mesh* mesh, dg_tiles* out);
/* Sets the budgets (the times are ignored; volume budgets 1..DG_MAX_VOL_BUDGET,
 * mortar budgets 1..DG_MAX_MORTAR_BUDGET nodes, else DG_ERR_ARG) and rebuilds
 * the work lists; releases cached dg_advance graphs.  Synchronous.
 * Errors: DG_ERR_ARG (null pointer, a budget out of range), DG_ERR_NOMEM,
 * DG_ERR_CUDA. */
dg_status dg_set_tiles(dg_mesh* mesh, const dg_tiles* in);

/* Adjoint (vector-Jacobian product) of the residual: out = (dR/dq)^T v at the
 * state q, on every mesh dg_residual accepts: affine or curved elements,
 * conforming, p-nonconforming (mortar) and boundary faces.  R = A Phi(q),
 * Phi the pointwise fluxes (contravariant volume flux, Roe at face and
 * mortar nodes) and A linear (GL derivative, surface lift, mortar
 * interpolation and L2 projection, -1/J): the kernels apply A^T and then
 * the flux Jacobians' transposes, taken exactly by forward-mode
 * differentiation of the same flux code (Dual numbers).  On curved or
 * Navier-Stokes mortars each side's flux (its own J a^dir on the mortar)
 * and the BR1 averages formed on the mortar are reversed the same way.
 * q, v, out: device state-layout arrays; out may not alias q or v.
 * Asynchronous.
 * Navier-Stokes adds the BR1 terms: the viscous flux's Jacobians in q and
 * in the gradient, the gradient's own transpose (GL derivative and lift) and
 * q-hat's (the interior average, the wall's q-hat(q_in)).
 * qinf_adj (device, 5 doubles, optional): accumulates the cotangent of the
 * far-field state q_inf (the Roe ghost and BR1's q-hat at far-field faces).
 * Errors: DG_ERR_ARG; DG_ERR_UNSUPPORTED (mortar batches whose adjoint
 * exceeds shared memory); DG_ERR_CUDA. */
dg_status dg_residual_vjp(dg_mesh* mesh, const double* q, const double* v, double* out, double* qinf_adj);

/* Force of the fluid on the boundary faces with tag `tag` (DG_BC_WALL: the
 * cylinder's drag and lift, Sec. 3.3):
 *   F = sum over those faces and their GL nodes of w_a w_b |J a^dir| (p n - tau n),
 * n the unit outward normal of the fluid element (into the body), p and tau
 * the pressure and viscous stress of the node's state and BR1 gradient
 * (tau = 0 for Euler).  force_dev: device double[3], written on the mesh
 * stream; the sum over the faces runs in a fixed order (deterministic).  Errors: DG_ERR_ARG
 * (null pointers, tag >= 0), DG_ERR_UNSUPPORTED (as dg_residual),
 * DG_ERR_NOMEM, DG_ERR_CUDA. */
dg_status dg_wall_force(dg_mesh* mesh, const double* q, int32_t tag, double* force_dev);
/* out = (dF/dq)^T lam (lam_dev: device double[3]), through the BR1 gradient
 * for Navier-Stokes; with scale_dev (device scalar) out += (*scale_dev) ...
 * Errors: as dg_residual_vjp. */
dg_status dg_wall_force_vjp(dg_mesh* mesh, const double* q, int32_t tag, const double* lam_dev, double* out,
                            const double* scale_dev);

/* Adjoint of one Williamson RK3 step (dg_rk_step) from the state q0 at the
 * step's start: lam <- (dq1/dq0)^T lam, with dt (the device scalar dt_dev)
 * held fixed.  The stage states are recomputed from q0; then, with
 * G_k = A_k G_{k-1} + dt R(Q_{k-1}) and Q_k = Q_{k-1} + B_k G_k reversed:
 * LG = B3 lam, lam += dt J(Q2)^T LG; LG = A3 LG + B2 lam, lam += dt J(Q1)^T LG;
 * LG = A2 LG + B1 lam, lam += dt J(q0)^T LG.  The mesh holds four states of
 * workspace.  qinf_adj (optional): accumulates the far-field state's
 * cotangent of the step.  Same support and errors as dg_residual_vjp. */
dg_status dg_rk_step_vjp(dg_mesh* mesh, const double* q0, const double* dt_dev, double* lam, double* qinf_adj);

/* Checkpoint and resume (the paper's runs restart from saved solutions,
 * Sec. 3.3): one host file with the element orders (they change with
 * adaptation), the time and the state, and an FNV-1a checksum.  Host memory
 * only, synchronous, no device involved.
 * dg_state_write: orders [n_elem][3], q_host in the state layout of those
 *   orders (dg_count_nodes nodes).
 * dg_state_info: n_elem, n_nodes and t of a file (each output optional).
 * dg_state_read: orders (host [n_elem][3]) and q_host (host, 5 n_nodes) of a
 *   file holding n_elem elements; t optional.
 * Errors: DG_ERR_ARG for bad arguments, an unreadable or unwritable path, a
 * wrong magic or version, a size mismatch, a truncated or longer file, or a
 * checksum mismatch. */
dg_status dg_state_write(const char* path, int32_t n_elem, const int32_t* orders, const double* q_host, double t);
dg_status dg_state_info(const char* path, int32_t* n_elem, int64_t* n_nodes, double* t);
dg_status dg_state_read(const char* path, int32_t n_elem, int32_t* orders, double* q_host, double* t);

/* Bounds-checking build (libdg compiled with -DDG_BOUNDS_CHECK; the
 * release build returns DG_ERR_UNSUPPORTED here).  Every kernel checks the
 * indices it reads from the mesh's work lists before it uses them (work items
 * and their element lists, face records, mortar batches and their faces, tau
 * sweep groups) and skips a unit whose indices are out of range, setting the
 * sticky DG_ERR_INDEX that dg_get_error reports (it takes precedence over
 * DG_ERR_NONPHYSICAL).
 * dg_debug_set_index overwrites one entry of a work list on the device, so
 * that tests can plant a bad index: list DG_LIST_VOLUME_ELEMENTS (element list
 * of the volume tiles, n_elem entries), DG_LIST_TAU_ELEMENTS (element list of
 * the tau tiles, n_elem), DG_LIST_FACE_LEFT (the left element of face record
 * i) or DG_LIST_MORTAR_FACES (entry i of the mortar faces' [L, R, dir]
 * triples).  old_value (optional) receives the entry's previous value.
 * Synchronous.  Errors: DG_ERR_ARG (null mesh, unknown list, i out of range),
 * DG_ERR_UNSUPPORTED (release build), DG_ERR_CUDA. */
enum { DG_LIST_VOLUME_ELEMENTS = 0, DG_LIST_TAU_ELEMENTS = 1, DG_LIST_FACE_LEFT = 2, DG_LIST_MORTAR_FACES = 3 };
dg_status dg_debug_set_index(dg_mesh* mesh, int32_t list, int64_t i, int32_t value, int32_t* old_value);

/* Kernel kinds for dg_profile_read. */
enum {
  DG_KERNEL_FACE_FLUX = 0,   /* Roe (+ BR1 viscous) numerical flux on conforming and boundary faces */
  DG_KERNEL_FACE_QHAT = 1,   /* BR1 q-hat per face (Navier-Stokes) */
  DG_KERNEL_GRADIENT = 2,    /* BR1 gradient (Navier-Stokes) */
  DG_KERNEL_VOLUME = 3,      /* volume residual + surface lift (+ fused RK3 stage) */
  DG_KERNEL_MAX_DT = 4,      /* CFL reduction and its finalisation (two launches) */
  DG_KERNEL_TAU = 5,         /* isolated tau sweep */
  DG_KERNEL_TAU_COMBINE = 6, /* non-isolated tau, per sweep entry */
  DG_KERNEL_PROJECT = 7,     /* order projection / restriction */
  DG_KERNEL_SELECT = 8,      /* order selection and degree-jump sweeps */
  DG_KERNEL_EXTRAP = 9,      /* truncation-error extrapolation */
  DG_KERNEL_MORTAR = 10,     /* p-nonconforming faces: mortar interpolation, Roe, L2 projection */
  DG_KERNEL_ADJOINT = 11,    /* residual / RK3 vector-Jacobian products */
  DG_KERNEL_KINDS = 12
};

/* Per-kernel timing with CUDA events recorded on the mesh stream around
 * every launch while enabled (on != 0 resets the totals).  Off by default.
 * Errors: DG_ERR_ARG (null mesh). */
dg_status dg_profile_enable(dg_mesh* mesh, int on);
/* Synchronises the stream and returns, for one kernel kind, the summed
 * event-measured duration (ms) and the number of timed launches since
 * profiling was enabled (host outputs; either may be NULL).
 * Errors: DG_ERR_ARG (null mesh, kernel outside 0..DG_KERNEL_KINDS-1),
 * DG_ERR_CUDA. */
dg_status dg_profile_read(dg_mesh* mesh, int kernel, double* total_ms, int64_t* launches);
/* Number of kernels the library has launched on this mesh since creation
 * (host output).  Errors: DG_ERR_ARG (null pointer). */
dg_status dg_launch_count(const dg_mesh* mesh, int64_t* launches);

/* Synchronises the mesh stream; returns and clears the sticky device error
 * (DG_OK if none): DG_ERR_NONPHYSICAL or, in the bounds-checking build,
 * DG_ERR_INDEX; DG_ERR_ARG for a null mesh, DG_ERR_CUDA if the
 * synchronisation fails. */
dg_status dg_get_error(dg_mesh* mesh);
/* A static description of a status code ("unknown status" for others). */
const char* dg_status_str(dg_status s);

#ifdef __cplusplus
}
#endif
#endif /* DG_H */
