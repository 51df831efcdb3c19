// dg_internal.h -- internal types of libdg (not part of the C ABI).
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <array>
#include <vector>

#include "../../include/dg.h"

#define DG_NV 5
#define DG_NP1 (DG_MAX_ORDER + 1)

// ---------------------------------------------------------------------------
// Basis tables (1D, orders 1..DG_MAX_ORDER), built on the host in basis.cpp
// and uploaded once per device into one buffer, FP64 and FP32 copies.
// ---------------------------------------------------------------------------
struct BasisOffsets {
  int D[DG_NP1];                 // D[N]: (N+1)x(N+1) GL derivative matrix
  int W[DG_NP1];                 // W[N]: N+1 GL weights
  int I[DG_NP1][DG_NP1];         // I[f][t]: (t+1)x(f+1) interpolation f -> t
  int P[DG_NP1][DG_NP1];         // P[f][t]: (t+1)x(f+1) L2 projection f -> t (t <= f)
  int X[DG_NP1];                 // X[N]: GL nodes
  int total;
};

namespace dgb {
void gl_nodes_weights(int N, double* x, double* w);
void build_tables(BasisOffsets* off, std::vector<double>* data);
// host helpers used by mesh construction
void deriv_matrix(int N, double* D);
void interp_matrix(const double* xf, int nf, const double* xt, int nt, double* I);
}  // namespace dgb

// ---------------------------------------------------------------------------
// Kernel-side views
// ---------------------------------------------------------------------------
struct DevPhys {
  int eqs;
  double gamma, mu, Pr, Rgas, kappa;
  double kappa_R;          // kappa / Rgas: the heat flux is kappa_R (grad p - (p/rho) grad rho) / rho
  double qinf[DG_NV];
};

// A face processed by the face kernels (one warp each).
struct FaceRec {
  int32_t L;       // element on the -xi_dir side (its face 2*dir+1), or the boundary element
  int32_t R;       // element on the +xi_dir side (its face 2*dir), or a DG_BC_* tag (< 0)
  int32_t face;    // interior: dir (0..2); boundary: the element's face (0..5)
  int32_t kind;    // 0 conforming interior, 1 mortar interior, 2 boundary
};

// Volume work item: `count` elements of one order triple, elist[first..first+count).
struct WorkItem {
  int32_t first, count;
  int32_t n1, n2, n3;
};

struct dg_mesh_impl;

// size classes of the tuned tile budgets: elements by node count, mortars by
// mortar nodes (<= 27 / 125 / 343 / more; <= 9 / 25 / 49 / more)
constexpr int kSizeClasses = DG_SIZE_CLASSES;
inline int elem_size_class(int n) { return n <= 27 ? 0 : n <= 125 ? 1 : n <= 343 ? 2 : 3; }
inline int mortar_size_class(int nm) { return nm <= 9 ? 0 : nm <= 25 ? 1 : nm <= 49 ? 2 : 3; }

// shared memory (doubles) of a batch of `count` mortar faces of one shape:
// the affine Euler kernel, and the general (curved or Navier-Stokes) kernels
size_t dg_mortar_smem_doubles(int count, int la, int lb, int ra, int rb);
size_t dg_mortar_general_smem_doubles(int count, int la, int lb, int ra, int rb, bool ns);

// per-kernel timing / launch counting hooks (capi.cpp), called by the launchers
void dg_prof_begin(dg_mesh_impl* m, int kernel_id, int n_launches);
void dg_prof_end(dg_mesh_impl* m, int kernel_id);

// kernels.cu launchers (all on mesh->stream)
namespace dgk {
void upload_basis(int device, const BasisOffsets& off, const std::vector<double>& data, const double** d64,
                  const float** d32);
cudaError_t face_flux(dg_mesh_impl* m, const double* q, const double* grad, bool isolated);
// the face fluxes of an RK stage: p-nonconforming and conforming interior
// faces of affine Euler meshes read the face traces of q from m->d_trace when
// trace_valid (the previous stage's volume kernel wrote them), else gather them
cudaError_t face_flux_rk(dg_mesh_impl* m, const double* q, bool trace_valid);
cudaError_t face_qhat(dg_mesh_impl* m, const double* q);
cudaError_t gradient(dg_mesh_impl* m, const double* q, double* grad, bool isolated);
cudaError_t volume(dg_mesh_impl* m, const double* q, const double* grad, double* r, bool isolated, int rk_stage,
                   double* q_io, double* g_io, const double* dt_dev);
cudaError_t max_dt(dg_mesh_impl* m, const double* q, double cfl, double* dt_dev);
cudaError_t tau_isolated(dg_mesh_impl* m, const double* q, const double* r_p, const int32_t* d_sweep, int n_sweep,
                         bool fp32, bool accumulate, void* map_new, void* map_trad);
cudaError_t tau_combine(dg_mesh_impl* m, dg_mesh_impl* coarse, const double* r_p, const double* r_c, int s,
                        int n_sweep, const int32_t* h_sweep, bool fp32, bool accumulate, void* map_new,
                        void* map_trad);
// mode 0: interpolate up / L2-project down (set_orders); mode 1: interpolate (restriction)
cudaError_t project_orders(dg_mesh_impl* m, const int32_t* d_new_orders, const int64_t* d_new_off,
                           const double* q_old, double* q_new, int mode);
// shared memory (dynamic + static bytes) of the isolated sweep's largest
// class, each class in the layout it runs with on a device offering `limit`
// bytes per block (the compact layout where the other does not fit)
size_t tau_smem_bytes(dg_mesh_impl* m, bool fp32, int limit);
// CFL reduction only: *bits = max over nodes of the inverse time-step scale
// (as the bit pattern of a non-negative double)
cudaError_t max_dt_bits(dg_mesh_impl* m, const double* q, unsigned long long* bits);
// adjoint: out = J(q)^T v, or out += (*scale) J(q)^T v (Euler, straight-sided elements)
cudaError_t residual_vjp(dg_mesh_impl* m, const double* q, const double* v, double* out, const double* scale,
                         bool accumulate, double* qinf_adj);
// force of the fluid on the boundary faces of a tag (device F[3]) and its
// vector-Jacobian product: out = (dF/dq)^T lam, or out += (*scale) ... (scale non-null)
cudaError_t wall_force(dg_mesh_impl* m, const double* q, int tag, double* F);
cudaError_t wall_force_vjp(dg_mesh_impl* m, const double* q, int tag, const double* lam, double* out,
                           const double* scale);
size_t mortar_adj_smem_max(dg_mesh_impl* m);
// y = a y + b x
cudaError_t axpby(dg_mesh_impl* m, double* y, const double* x, double a, double b, int64_t n);
}  // namespace dgk

// One metric job of the device construction (rebuild.cu): element e at
// orders (n1-1, n2-1, n3-1), written at out (doubles) as fields
// [J a^i_d (9), J, with 11 fields also 1/J][n].
struct DgGeomJob {
  int32_t e, n1, n2, n3;
  int64_t out;
};
// Metrics of every job on the mesh's stream (out32: an FP32 copy of the
// fields, or null), from the lattices at m->d_geom; DG_ERR_ARG where a
// Jacobian is not positive.  Synchronous.
dg_status dg_device_metrics(dg_mesh_impl* m, const std::vector<DgGeomJob>& jobs, int fields, double* out,
                            float* out32);

// The order-dependent lists built on the device (rebuild.cu): the mesh's
// d_off / d_soff, the warp-list faces d_faces and d_fnodes are set; the host
// copies below feed the tiling of buckets and shape groups.
struct DgDeviceLists {
  std::vector<int64_t> off, soff;                  // node and face-node offsets
  std::vector<int32_t> bucket_key, bucket_elems;   // elements sorted by order triple (key ((N1-1) 8 + N2-1) 8 + N3-1)
  std::vector<int32_t> mfaces;                     // batched faces [L, R, dir], sorted by shape, then direction
  std::vector<int32_t> msig;                       // their shapes ((la 16 + lb) 16 + ra) 16 + rb
  int n_conf = 0, n_mortar = 0, n_bnd = 0;         // conforming interior, p-nonconforming, boundary faces
};
dg_status dg_device_lists(dg_mesh_impl* m, bool batch_conforming, DgDeviceLists* out);

// work-list (re)builders with the mesh's tile budgets (capi.cpp)
dg_status build_volume_items(dg_mesh_impl* m);
dg_status build_mortar_batches(dg_mesh_impl* m);

// releases the dg_advance graphs and capture stream of a mesh
void dg_advance_release(dg_mesh_impl* m);

// one RK3 step (capi.cpp); trace_valid: the mesh's face-trace buffer holds the
// traces of q (the step before ran on the same q and nothing changed it)
dg_status rk_step_impl(dg_mesh_impl* m, double* q, double* g, const double* dt_dev, bool trace_valid);

// ---------------------------------------------------------------------------
// The mesh
// ---------------------------------------------------------------------------
struct dg_mesh_impl {
  int device = 0;
  cudaStream_t stream = nullptr;
  int n_elem = 0, G = 1;
  int64_t n_nodes = 0;
  DevPhys phys{};
  bool affine = true;       // every element a parallelepiped: metrics per element
  bool axis = false;        // affine and every J a^i parallel to e_i (axis-aligned box)
  int max_order = 1;        // max over elements and directions
  bool faces_unsupported = false;  // face-coupled calls refused (mortars whose shared memory exceeds the device's)
  bool general_mortars = false;    // mortars on a curved or Navier-Stokes mesh (own-normal flux per side)

  // host copies (for rebuilds and coarse meshes)
  std::vector<double> h_geom;
  double* d_geom = nullptr;        // curved meshes: the geometry lattices on the device (metric construction)
  bool device_build = false;       // the order-dependent lists and metrics are built on the device (rebuild.cu)
  std::vector<int32_t> h_nbr, h_ord;
  std::vector<int64_t> h_off, h_soff;
  std::vector<double> h_xyz;       // node coordinates (state-order [d][node] per element)

  // device data
  int32_t* d_ord = nullptr;        // [e][3]
  int32_t* d_nbr = nullptr;        // [e][6]
  int64_t* d_off = nullptr;        // [e+1] node offsets
  int64_t* d_soff = nullptr;       // [e+1] surface (face-node) offsets, 6 faces per element
  double* d_metric = nullptr;      // affine: [e][16] (J a^i_d, J, 1/J, pad); curved: [11][n] at 11*off_e
  float* d_metric32 = nullptr;     // affine: FP32 copy for the FP32 tau sweep
  double* d_surf = nullptr;        // [5 * soff_total] numerical contravariant flux per element face node
  double* d_trace = nullptr;       // affine Euler meshes: [5 * soff_total] the state at every element face node,
                                   // written by each RK stage's volume kernel for the next stage's mortar fluxes
  double* d_surfq = nullptr;       // NS: [15 * soff_total] BR1 q-hat * J a^dir
  double* d_grad = nullptr;        // NS: [15 * n_nodes] gradient [c][v][node]
  double* d_xyz = nullptr;         // lazily uploaded coordinates
  FaceRec* d_faces = nullptr;      // conforming and boundary faces
  int32_t* d_fnodes = nullptr;     // (face, node) pairs of those faces, one thread each
  int n_fnodes = 0;
  int n_faces = 0, n_face_conf = 0, n_face_mortar = 0, n_face_bnd = 0;
  int32_t* d_mfaces = nullptr;     // p-nonconforming faces [L, R, dir], grouped by shape signature
  int n_mfaces = 0;
  int32_t* d_mbatches = nullptr;   // mortar batches [first, count, la, lb, ra, rb]
  int n_mbatches = 0;
  size_t mortar_smem = 0;          // doubles of shared memory of the largest batch
  WorkItem* d_items = nullptr;     // tiles of <= 256 nodes (tau sweep)
  int32_t* d_elist = nullptr;
  int n_items = 0;
  // volume / gradient / CFL tiles, with a node budget per element-size class
  // (dg_autotune), and the mortar batches' budget per mortar-size class
  int vol_budget[kSizeClasses] = {256, 256, 256, 256};
  int mortar_budget[kSizeClasses] = {256, 256, 256, 256};
  WorkItem* d_vitems = nullptr;
  int32_t* d_velist = nullptr;
  int n_vitems = 0;
  std::vector<WorkItem> h_vitems;
  std::vector<std::array<int, 3>> h_bucket_key;    // order triples
  std::vector<std::vector<int32_t>> h_buckets;     // their elements
  struct MGroup { int la, lb, ra, rb; std::vector<int32_t> faces; };
  std::vector<MGroup> h_mgroups;                   // batched faces [L, R, dir] by shape, sorted by direction
  std::vector<int32_t> h_mbatches;                 // [first, count, la, lb, ra, rb] per batch, as uploaded
  unsigned* d_err = nullptr;       // sticky error word
  double* d_scratch = nullptr;     // dt reduction
  // tau geometry bank (curved meshes): metrics at every coarse order N <= P
  double* d_taugeo = nullptr;
  float* d_taugeo32 = nullptr;
  int64_t* d_taugeo_off = nullptr;

  const double* basis64 = nullptr;
  const float* basis32 = nullptr;
  BasisOffsets boff{};

  std::vector<dg_mesh_impl*> coarse;   // cached non-isolated coarse meshes (by sweep entry)
  std::vector<int32_t> coarse_key;     // their sweep orders, 3 per entry
  double* d_rp = nullptr;              // tau: R^P scratch (full R^P non-isolated, isolated R^P FP64 sweep)
  float* d_rp32 = nullptr;             // tau: isolated R^P scratch of the FP32 sweep
  struct TauClass { int32_t* d_list; int n; int S; };
  std::vector<TauClass> tau_classes;   // work items grouped by tile size (shared-memory size class)
  std::vector<TauClass> vol_classes;   // the same items split in two for the volume kernels (<= 400 nodes, larger)
  // isolated sweep units for the last sweep: (item, group) per class, groups of
  // entries sharing (N2, N3) [N2, N3, first, count], entries [sweep index, N1]
  std::vector<int32_t*> tau_units;
  std::vector<int> tau_n_units;
  std::vector<int> tau_n_shared;       // units of a class holding two groups or more (the xi3 restriction shared)
  std::vector<int32_t*> tau_units_split;   // the same units with one group each (the compact FP64 layout)
  std::vector<int> tau_n_units_split;
  std::vector<int> tau_last_units, tau_last_shared;   // per class, the units the last isolated sweep ran
  int tau_unit_mode = DG_TAU_UNITS_AUTO;
  int32_t* d_tgroups = nullptr;
  int32_t* d_tgentries = nullptr;
  int n_tgroups = 0, n_tgentries = 0;
  std::vector<WorkItem> h_items;
  double* d_qc = nullptr;              // coarse mesh: restricted state scratch
  double* d_rc = nullptr;              // coarse mesh: coarse residual scratch
  int32_t* d_sweep = nullptr;          // device copy of the last sweep
  std::vector<int32_t> h_sweep;

  // CUDA-event timing per kernel kind (dg_profile_*), and the launch counter
  bool prof_on = false;
  struct ProfPair { int id; cudaEvent_t a, b; };
  std::vector<ProfPair> prof_pending;
  std::vector<cudaEvent_t> prof_pool;
  cudaEvent_t prof_open = nullptr;
  double prof_ms[DG_KERNEL_KINDS] = {0};
  int64_t prof_n[DG_KERNEL_KINDS] = {0};
  int64_t launches = 0;

  // dg_advance: device block {cfl, t_end, dt, steps}, the capture stream and
  // the instantiated step batches, keyed by the caller's buffers
  double* d_adv = nullptr;
  // adjoint: trace cotangents per element face node (face-buffer layout) and
  // the RK3 step's workspace (stage states Q1, Q2 and the register's cotangent)
  double* d_sadj = nullptr;
  double* d_adjw = nullptr;
  // Navier-Stokes adjoint: gradient cotangents per element face node and per
  // node, the lifted q-hat's cotangent per element face node, a state scratch
  double* d_gadj = nullptr;
  double* d_lG = nullptr;
  double* d_lS = nullptr;
  double* d_adjt = nullptr;
  double* d_force = nullptr;   // wall force: one partial per warp-list face
  // dg_step_host: the device copies of its host buffers (state, RK register,
  // time, both maps of map_bytes each)
  double* d_hq = nullptr;
  double* d_hg = nullptr;
  double* d_ht = nullptr;
  void* d_hmap_new = nullptr;
  void* d_hmap_trad = nullptr;
  size_t hmap_bytes = 0;
  cudaStream_t cap_stream = nullptr;
  bool adv_warm = false;             // one eager step taken (kernel attributes set)
  struct AdvGraph { const void *q, *g, *t; int steps; cudaGraphExec_t exec; int64_t launches; };
  std::vector<AdvGraph> adv_graphs;
};

struct dg_mesh : dg_mesh_impl {};
