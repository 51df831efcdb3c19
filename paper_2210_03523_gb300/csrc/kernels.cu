// kernels.cu -- sm_103a kernels of libdg.
//
// Hot path (Sec. 2.1 DGSEM residual, Sec. 3 RK3, Sec. 2.3 tau sweep):
//   face_node_flux_kernel  Roe (+ BR1 viscous average) numerical flux, one
//                      thread per face node; p-nonconforming faces through
//                      mortars staged in shared memory (interpolate both
//                      traces up, Roe at mortar nodes, L2-project back).
//   face_qhat_kernel   BR1 q-hat * J a^dir on every face (Navier-Stokes).
//   gradient_kernel    BR1 gradient, strong form (Navier-Stokes).
//   volume_kernel      nodal + contravariant flux, sum-factorised GL
//                      derivative in three directions, surface lift,
//                      -(1/J) scaling, optionally the fused RK3 stage update.
//                      Elements of one order triple are batched per CTA
//                      (work items), all triples in one launch.
//   tau_kernel<T>      isolated tau sweep, one CTA per unit (a tile and the
//                      groups of sweep entries sharing (N2,N3) for one N3):
//                      restriction by sum-factorised interpolation (xi3 once
//                      per unit, xi2 once per group, xi1 per chunk of
//                      entries), coarse isolated residual, both tau forms,
//                      per-element maxima.
// FP64 throughout, except tau_kernel<float>.
#include <algorithm>
#include <atomic>
#include <cfloat>
#include <cstdio>
#include <cstring>
#include <map>
#include <type_traits>
#include <utility>

#include "dg_internal.h"

__constant__ BasisOffsets c_boff;

// Division by a small runtime divisor (1..kFdivMax) as a multiply-high and
// two shifts (Granlund and Montgomery, "Division by invariant integers using
// multiplication", 1994, the round-up method for full 32-bit dividends): the
// multiplier and shift of every divisor in constant memory, read by a warp
// whose divisor is uniform as one broadcast.  The tau sweep's index
// arithmetic spends its integer pipe on these divisions otherwise.
constexpr int kFdivMax = 1024;
__constant__ uint2 c_fdiv[kFdivMax + 1];

__device__ __forceinline__ int fdiv(int n, int d) {
  if (d > kFdivMax) return n / d;
  const uint2 c = c_fdiv[d];
  const uint32_t un = (uint32_t)n, t1 = __umulhi(c.x, un);
  return (int)((t1 + ((un - t1) >> (c.y ? 1u : 0u))) >> (c.y ? c.y - 1u : 0u));
}

namespace {

constexpr int kFaceWarps = 4;          // faces per CTA in the face kernels
constexpr int kVolThreads = 256;
// volume tiles' shared memory above which two CTAs, or one, fit an SM
constexpr size_t kVolThreeCtaBytes = 400 * 20 * sizeof(double), kVolTwoCtaBytes = 700 * 20 * sizeof(double);
constexpr int kTauChunk = 16;   // at most this many sweep entries share the two barriers of a tau chunk
constexpr int kTauBatchGroups = 16;    // (N2, N3) groups of one Euler tau batch at most
constexpr int kTauBatchEntries = 64;   // entries of a batch's table at most (a larger batch runs in pieces)
constexpr int kTauThreads = 128;
constexpr int kTauRefElems = 32;   // elements of a tau tile at most (tiles of <= 256 nodes, 8 nodes an element)
constexpr int kTauRefStride = 16;  // floats of one element's reference record

// ------------------------------------------------------------------ helpers
// offset (in face nodes) of face f inside an element's surface block
__device__ __forceinline__ int face_offset(int n1, int n2, int n3, int f) {
  int s0 = n2 * n3, s1 = n1 * n3, s2 = n1 * n2;
  int o = 0;
  if (f >= 1) o += s0;
  if (f >= 2) o += s0;
  if (f >= 3) o += s1;
  if (f >= 4) o += s1;
  if (f >= 5) o += s2;
  return o;
}

// volume node index of face node (a, b) on face f; (a, b) run over the
// two tangential directions in increasing order
__device__ __forceinline__ int face_vidx(int n1, int n2, int n3, int f, int a, int b) {
  int d = f >> 1, side = f & 1;
  int i, j, k;
  if (d == 0) { i = side ? n1 - 1 : 0; j = a; k = b; }
  else if (d == 1) { j = side ? n2 - 1 : 0; i = a; k = b; }
  else { k = side ? n3 - 1 : 0; i = a; j = b; }
  return i + n1 * (j + n2 * k);
}


// Metric record: field m of element e at node p.  Fields 0..8: J a^i_d
// (index 3i+d); 9: J; 10: 1/J; affine records also 11..13: |J a^i|.
// Affine meshes: one record of kAffStride doubles per element; curved
// meshes: [kCurvedFields][n] per element at kCurvedFields * off_e.
constexpr int kAffStride = 16;
constexpr int kCurvedFields = 11;

template <bool AFFINE>
__device__ __forceinline__ double metric(const double* M, int e, int64_t off, int n, int p, int m) {
  if (AFFINE) return __ldg(M + kAffStride * (int64_t)e + m);
  return __ldg(M + kCurvedFields * off + (int64_t)m * n + p);
}

struct Prim {
  double rho, ir, u[3], p;
};

__device__ __forceinline__ Prim primitive(double gm1, const double q[5]) {
  Prim s;
  s.rho = q[0];
  s.ir = 1.0 / q[0];
  s.u[0] = q[1] * s.ir;
  s.u[1] = q[2] * s.ir;
  s.u[2] = q[3] * s.ir;
  s.p = gm1 * (q[4] - 0.5 * (q[1] * s.u[0] + q[2] * s.u[1] + q[3] * s.u[2]));
  return s;
}

// Forward-mode dual number (value, derivative along one seed direction): the
// adjoint kernels differentiate the flux functions below exactly by running
// them on Dual, one input component seeded at a time (Jacobian columns).
struct Dual {
  double v, d;
};
__device__ __forceinline__ Dual mkd(double v) { return {v, 0.0}; }
__device__ __forceinline__ Dual operator+(Dual a, Dual b) { return {a.v + b.v, a.d + b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, Dual b) { return {a.v - b.v, a.d - b.d}; }
__device__ __forceinline__ Dual operator-(Dual a) { return {-a.v, -a.d}; }
__device__ __forceinline__ Dual operator*(Dual a, Dual b) { return {a.v * b.v, a.v * b.d + a.d * b.v}; }
__device__ __forceinline__ Dual operator/(Dual a, Dual b) {
  const double r = 1.0 / b.v;
  return {a.v * r, (a.d - a.v * r * b.d) * r};
}
__device__ __forceinline__ Dual operator+(Dual a, double b) { return {a.v + b, a.d}; }
__device__ __forceinline__ Dual operator+(double a, Dual b) { return {a + b.v, b.d}; }
__device__ __forceinline__ Dual operator-(Dual a, double b) { return {a.v - b, a.d}; }
__device__ __forceinline__ Dual operator-(double a, Dual b) { return {a - b.v, -b.d}; }
__device__ __forceinline__ Dual operator*(Dual a, double b) { return {a.v * b, a.d * b}; }
__device__ __forceinline__ Dual operator*(double a, Dual b) { return {a * b.v, a * b.d}; }
__device__ __forceinline__ Dual operator/(Dual a, double b) { return {a.v / b, a.d / b}; }
__device__ __forceinline__ Dual operator/(double a, Dual b) {
  const double r = 1.0 / b.v;
  return {a * r, -a * r * r * b.d};
}
__device__ __forceinline__ Dual& operator+=(Dual& a, Dual b) { return a = a + b; }
__device__ __forceinline__ Dual& operator-=(Dual& a, Dual b) { return a = a - b; }
__device__ __forceinline__ Dual& operator*=(Dual& a, double b) { return a = a * b; }
__device__ __forceinline__ bool operator>(Dual a, double b) { return a.v > b; }
// the two nonlinear primitives of the fluxes, on double and on Dual
__device__ __forceinline__ double rsq(double x) { return rsqrt(x); }
__device__ __forceinline__ Dual rsq(Dual x) {
  const double r = rsqrt(x.v);
  return {r, -0.5 * r * r * r * x.d};
}
__device__ __forceinline__ double absval(double x) { return fabs(x); }
__device__ __forceinline__ Dual absval(Dual x) { return x.v < 0.0 ? Dual{-x.v, -x.d} : x; }
__device__ __forceinline__ double val(double x) { return x; }
__device__ __forceinline__ double val(Dual x) { return x.v; }

// Roe's approximate Riemann solver: flux through the unit normal n from qL
// (behind) to qR (ahead).  AX >= 0: the normal is the unit vector e_AX (axis
// aligned faces), n is not read.  sqrt(rho) and 1/rho come from one rsqrt,
// as do the Roe sound speed and its inverse square.  S: double, or Dual for
// the adjoint's Jacobian columns.
template <int AX>
__device__ __forceinline__ double ncomp(const double n[3], int c) {
  return AX >= 0 ? (c == AX ? 1.0 : 0.0) : n[c];
}

template <int AX, typename S = double>
__device__ void roe_t(double gamma, const S qL[5], const S qR[5], const double n[3], S f[5], double hs) {
  const double gm1 = gamma - 1.0, hgm1 = 0.5 * gm1;
  const S rsL = rsq(qL[0]), rsR = rsq(qR[0]);
  const S sL = qL[0] * rsL, sR = qR[0] * rsR;      // sqrt(rho)
  const S irL = rsL * rsL, irR = rsR * rsR;        // 1/rho
  S uL[3], uR[3];
  for (int c = 0; c < 3; ++c) {
    uL[c] = qL[1 + c] * irL;
    uR[c] = qR[1 + c] * irR;
  }
  // p = gm1 E - (gm1/2) m.u
  const S pL = gm1 * qL[4] - hgm1 * (qL[1] * uL[0] + qL[2] * uL[1] + qL[3] * uL[2]);
  const S pR = gm1 * qR[4] - hgm1 * (qR[1] * uR[0] + qR[2] * uR[1] + qR[3] * uR[2]);
  const S eL = qL[4] + pL, eR = qR[4] + pR;        // rho H
  const S HL = eL * irL, HR = eR * irR;
  // Roe averages with the weights sqrt(rho_L,R) / (sqrt(rho_L) + sqrt(rho_R))
  const S is = 1.0 / (sL + sR);
  const S wL = sL * is, wR = sR * is;
  S ut[3];
  for (int c = 0; c < 3; ++c) ut[c] = wL * uL[c] + wR * uR[c];
  const S Ht = wL * HL + wR * HR;
  const S rt = sL * sR;
  const S q2 = ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2];
  const S c2 = gm1 * (Ht - 0.5 * q2);
  const S rc = rsq(c2);
  const S ct = c2 * rc, ic2 = rc * rc, hic2 = 0.5 * ic2;
  S unL, unR, utn, mL, mR;
  if (AX >= 0) {
    unL = uL[AX];
    unR = uR[AX];
    utn = ut[AX];
    mL = qL[1 + AX];   // rho u_n: the normal momentum itself
    mR = qR[1 + AX];
  } else {
    unL = uL[0] * n[0] + uL[1] * n[1] + uL[2] * n[2];
    unR = uR[0] * n[0] + uR[1] * n[1] + uR[2] * n[2];
    utn = ut[0] * n[0] + ut[1] * n[1] + ut[2] * n[2];
    mL = qL[0] * unL;
    mR = qR[0] * unR;
  }
  const S dun = unR - unL, dp = pR - pL, dr = qR[0] - qL[0];
  const S rcd = rt * ct * dun;
  const S a1 = (dp - rcd) * hic2;
  const S a5 = (dp + rcd) * hic2;
  const S a2 = dr - dp * ic2;
  const S l1a1 = absval(utn - ct) * a1, l5a5 = absval(utn + ct) * a5, l2 = absval(utn);
  const S s15 = l1a1 + l5a5, d15 = (l5a5 - l1a1) * ct;
  // tangential velocity jump; on an axis normal its normal component is exactly zero
  S dut[3], utdut{};
  for (int c = 0; c < 3; ++c) {
    if (AX >= 0) {
      dut[c] = c == AX ? S{} : uR[c] - uL[c];
      if (c != AX) utdut += ut[c] * dut[c];
    } else {
      dut[c] = (uR[c] - uL[c]) - dun * n[c];
      utdut += ut[c] * dut[c];
    }
  }
  f[0] = hs * ((mL + mR) - (s15 + l2 * a2));
  for (int c = 0; c < 3; ++c) {
    const double nc = ncomp<AX>(n, c);
    S phys = mL * uL[c] + mR * uR[c];
    S inner = a2 * ut[c];
    if (AX < 0 || c != AX) inner += rt * dut[c];   // dut[AX] = 0 on an axis normal
    S diss = s15 * ut[c] + l2 * inner;
    if (AX < 0 || c == AX) {
      phys += (pL + pR) * nc;
      diss += d15 * nc;
    }
    f[1 + c] = hs * (phys - diss);
  }
  const S physE = unL * eL + unR * eR;
  const S dissE = s15 * Ht + d15 * utn + l2 * (a2 * 0.5 * q2 + rt * utdut);
  f[4] = hs * (physE - dissE);
}

// Roe on a face of direction dir times the face area |J a^dir|: the
// axis-aligned variant when the mesh is an axis-aligned box (normal e_dir),
// else the general one.  The area rides on the flux's own factor 1/2 (0.5
// area is exact), which gives the bits of (0.5 (...)) * area with five
// multiplications fewer.
template <bool AXIS>
__device__ __forceinline__ void roe_face(double gamma, int dir, const double qL[5], const double qR[5],
                                         const double n[3], double area, double f[5]) {
  const double hs = 0.5 * area;
  if (AXIS) {
    if (dir == 0) roe_t<0>(gamma, qL, qR, n, f, hs);
    else if (dir == 1) roe_t<1>(gamma, qL, qR, n, f, hs);
    else roe_t<2>(gamma, qL, qR, n, f, hs);
  } else {
    roe_t<-1>(gamma, qL, qR, n, f, hs);
  }
}

// Navier-Stokes viscous flux for all three directions: fv[d][v].
// g[v*3+c] = d q_v / d x_c.
__device__ void viscous(const DevPhys& ph, const double q[5], const double g[15], double fv[3][5]) {
  double gm1 = ph.gamma - 1.0;
  Prim s = primitive(gm1, q);
  // dT = R grad T = (grad p - (p/rho) grad rho) / rho; the heat flux is (kappa/R) dT
  const double pir = s.p * s.ir;
  double du[3][3], dT[3];
  double half_u2 = 0.5 * (s.u[0] * s.u[0] + s.u[1] * s.u[1] + s.u[2] * s.u[2]);
  for (int c = 0; c < 3; ++c) {
    for (int i = 0; i < 3; ++i) du[i][c] = (g[(1 + i) * 3 + c] - s.u[i] * g[c]) * s.ir;
    double dpc = gm1 * (g[12 + c] - (s.u[0] * g[3 + c] + s.u[1] * g[6 + c] + s.u[2] * g[9 + c]) + half_u2 * g[c]);
    dT[c] = (dpc - pir * g[c]) * s.ir;
  }
  double div = du[0][0] + du[1][1] + du[2][2];
  for (int d = 0; d < 3; ++d) {
    double tau[3];
    for (int i = 0; i < 3; ++i) tau[i] = ph.mu * (du[i][d] + du[d][i]) - (i == d ? (2.0 / 3.0) * ph.mu * div : 0.0);
    fv[d][0] = 0.0;
    fv[d][1] = tau[0];
    fv[d][2] = tau[1];
    fv[d][3] = tau[2];
    fv[d][4] = s.u[0] * tau[0] + s.u[1] * tau[1] + s.u[2] * tau[2] + ph.kappa_R * dT[d];
  }
}

__device__ __forceinline__ void bc_ghost(const DevPhys& ph, int tag, const double qi[5], double qg[5]) {
  if (tag == DG_BC_WALL) {
    qg[0] = qi[0]; qg[1] = -qi[1]; qg[2] = -qi[2]; qg[3] = -qi[3]; qg[4] = qi[4];
  } else {
    for (int v = 0; v < 5; ++v) qg[v] = ph.qinf[v];
  }
}

__device__ __forceinline__ void bc_qhat(const DevPhys& ph, int tag, const double qi[5], double qh[5]) {
  if (tag == DG_BC_WALL) {
    qh[0] = qi[0]; qh[1] = 0.0; qh[2] = 0.0; qh[3] = 0.0;
    qh[4] = qi[4] - 0.5 * (qi[1] * qi[1] + qi[2] * qi[2] + qi[3] * qi[3]) / qi[0];
  } else {
    for (int v = 0; v < 5; ++v) qh[v] = ph.qinf[v];
  }
}

struct MeshView {
  const int32_t* ord;
  const int64_t* off;
  const int64_t* soff;
  const double* metric;
  DevPhys ph;
  int n_elem;
  int64_t n_nodes;
  int64_t n_surf;    // element-face nodes (the face buffers' length)
  unsigned* err;     // the sticky error word
};

// ------------------------------------------------ bounds-checking build
// Built with -DDG_BOUNDS_CHECK, every kernel checks the indices it reads from
// the mesh's work lists before it uses them: work items and their element
// lists, face records and mortar batches.  A failed check sets bit 1 of the
// sticky error word (dg_get_error: DG_ERR_INDEX) and the kernel skips that
// unit of work; nothing out of range is read or written.  The release build
// compiles the checks away.
__device__ __forceinline__ void flag_index(const MeshView& m) { atomicOr(m.err, 2u); }

// element e exists, has orders (N1,N2,N3) and its nodes lie inside the state
__device__ __forceinline__ bool elem_fits(const MeshView& m, int e, int N1, int N2, int N3) {
  if ((unsigned)e >= (unsigned)m.n_elem) return false;
  if (m.ord[3 * e] != N1 || m.ord[3 * e + 1] != N2 || m.ord[3 * e + 2] != N3) return false;
  const int n1 = N1 + 1, n2 = N2 + 1, n3 = N3 + 1;
  const int64_t o = m.off[e], so = m.soff[e];
  return o >= 0 && o + (int64_t)n1 * n2 * n3 <= m.n_nodes && so >= 0 &&
         so + 2 * (int64_t)(n2 * n3 + n1 * n3 + n1 * n2) <= m.n_surf;
}

__device__ __forceinline__ unsigned dynamic_smem_bytes() {
  unsigned r;
  asm("mov.u32 %0, %%dynamic_smem_size;" : "=r"(r));
  return r;
}

// Work item wi of a block-uniform loop into w; false: skip it.  In the
// checking build every thread of the block must call it (a block-wide vote);
// smem_per_node: the doubles of dynamic shared memory the kernel lays out per
// tile node (0: none), checked against the launch's allocation.
__device__ __forceinline__ bool take_item(const MeshView& m, const WorkItem* items, int wi, int n_items,
                                          const int32_t* elist, int smem_per_node, WorkItem& w) {
#ifdef DG_BOUNDS_CHECK
  bool bad = (unsigned)wi >= (unsigned)n_items;
  if (!bad) {
    w = items[wi];
    bad = w.count < 1 || w.first < 0 || w.first > m.n_elem - w.count || w.n1 < 1 || w.n1 > DG_MAX_ORDER ||
          w.n2 < 1 || w.n2 > DG_MAX_ORDER || w.n3 < 1 || w.n3 > DG_MAX_ORDER;
    if (!bad && smem_per_node > 0)
      bad = (uint64_t)w.count * (w.n1 + 1) * (w.n2 + 1) * (w.n3 + 1) * smem_per_node * sizeof(double) >
            dynamic_smem_bytes();
    for (int el = threadIdx.x; !bad && el < w.count; el += blockDim.x)
      bad = !elem_fits(m, elist[w.first + el], w.n1, w.n2, w.n3);
  }
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) flag_index(m);
  return !bad;
#else
  (void)n_items;
  (void)elist;
  (void)smem_per_node;
  w = items[wi];
  return true;
#endif
}

// a face record's elements, tag and face number (warp-uniform)
__device__ __forceinline__ bool bad_face(const MeshView& m, const FaceRec& f) {
#ifdef DG_BOUNDS_CHECK
  bool bad = (unsigned)f.L >= (unsigned)m.n_elem || f.kind < 0 || f.kind > 2;
  if (!bad) bad = !elem_fits(m, f.L, m.ord[3 * f.L], m.ord[3 * f.L + 1], m.ord[3 * f.L + 2]);
  if (!bad && f.kind == 2) bad = (f.R != DG_BC_FARFIELD && f.R != DG_BC_WALL) || (unsigned)f.face >= 6u;
  else if (!bad)
    bad = (unsigned)f.R >= (unsigned)m.n_elem || (unsigned)f.face >= 3u ||
          !elem_fits(m, f.R, m.ord[3 * f.R], m.ord[3 * f.R + 1], m.ord[3 * f.R + 2]);
  if (bad) flag_index(m);
  return bad;
#else
  (void)m;
  (void)f;
  return false;
#endif
}

__device__ __forceinline__ void orders_of(const MeshView& m, int e, int& n1, int& n2, int& n3) {
  n1 = __ldg(m.ord + 3 * e) + 1;
  n2 = __ldg(m.ord + 3 * e + 1) + 1;
  n3 = __ldg(m.ord + 3 * e + 2) + 1;
}

// ------------------------------------------------------------- face kernels
struct FaceParams {
  MeshView m;
  const FaceRec* faces;
  int n_faces;
  const double* q;
  const double* grad;
  double* surf;
  const double* basis;
  int np_max;            // max order + 1 (mortar smem sizing)
  int warp_smem;         // doubles per warp
  const int2* fnodes;    // (face, node) of every face node, faces in order
  int n_fnodes;
};

template <bool AFFINE>
__device__ __forceinline__ void face_metric(const MeshView& m, int e, int n, int vi, int dir, double ja[3]) {
  int64_t o = AFFINE ? 0 : m.off[e];
  for (int c = 0; c < 3; ++c) ja[c] = metric<AFFINE>(m.metric, e, o, n, vi, 3 * dir + c);
}

__device__ __forceinline__ double unit_normal(const double ja[3], double nrm[3]) {
  const double a2 = ja[0] * ja[0] + ja[1] * ja[1] + ja[2] * ja[2];
  const double ia = rsqrt(a2);
  nrm[0] = ja[0] * ia;
  nrm[1] = ja[1] * ia;
  nrm[2] = ja[2] * ia;
  return a2 * ia;   // |J a|
}


// Numerical flux on the conforming interior (kind 0) and boundary (kind 2)
// faces, one thread per face node over the (face, node) list, so that faces
// of any size pack the warps (a warp per face left lanes idle on faces of
// fewer than 32 nodes, e.g. 7 x 2 on a P = (6,6,1) mesh).  Writes the
// contravariant numerical flux F* in the +xi_dir direction, |J a^dir| times
// Roe (minus the BR1 viscous average for Navier-Stokes), onto each side's own
// face grid.  AFFINE: J a^dir is the element record's constant; AXIS: it is
// aligned with e_dir.
constexpr int kFaceNodeThreads = 128;
template <bool AFFINE, bool AXIS, bool NS>
__global__ void __launch_bounds__(kFaceNodeThreads, 4) face_node_flux_kernel(FaceParams P) {
  const int g = blockIdx.x * kFaceNodeThreads + threadIdx.x;
  if (g >= P.n_fnodes) return;
  const int2 fp = P.fnodes[g];
#ifdef DG_BOUNDS_CHECK
  if ((unsigned)fp.x >= (unsigned)P.n_faces) {
    flag_index(P.m);
    return;
  }
#endif
  const FaceRec fr = P.faces[fp.x];
  if (bad_face(P.m, fr)) return;
  const MeshView& m = P.m;
  const double gamma = m.ph.gamma;
  const int p = fp.y;
  if (fr.kind == 2) {  // boundary face of element fr.L, face fr.face, tag fr.R
    const int e = fr.L, f = fr.face, tag = fr.R, dir = f >> 1, side = f & 1;
    int n1, n2, n3;
    orders_of(m, e, n1, n2, n3);
    const int n = n1 * n2 * n3;
    const int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3, nf = na * nb;
#ifdef DG_BOUNDS_CHECK
    if ((unsigned)p >= (unsigned)nf) {
      flag_index(m);
      return;
    }
#endif
    const int64_t o = m.off[e];
    double* out = P.surf + 5 * (m.soff[e] + face_offset(n1, n2, n3, f));
    const int vi = face_vidx(n1, n2, n3, f, p % na, p / na);
    double ja[3], nrm[3];
    face_metric<AFFINE>(m, e, n, vi, dir, ja);
    const double area = unit_normal(ja, nrm);
    double qi[5], qg[5], F[5];
    for (int v = 0; v < 5; ++v) qi[v] = P.q[5 * o + v * n + vi];
    bc_ghost(m.ph, tag, qi, qg);
    if (side) roe_face<AXIS>(gamma, dir, qi, qg, nrm, area, F);
    else roe_face<AXIS>(gamma, dir, qg, qi, nrm, area, F);
    if (NS) {
      double gr[15], fv[3][5];
      for (int v = 0; v < 5; ++v)
        for (int c = 0; c < 3; ++c) gr[v * 3 + c] = P.grad[15 * o + (c * 5 + v) * n + vi];
      viscous(m.ph, qi, gr, fv);
      for (int v = 1; v < 4; ++v) F[v] -= fv[0][v] * ja[0] + fv[1][v] * ja[1] + fv[2][v] * ja[2];
      if (tag != DG_BC_WALL) F[4] -= fv[0][4] * ja[0] + fv[1][4] * ja[1] + fv[2][4] * ja[2];
    }
    for (int v = 0; v < 5; ++v) out[v * nf + p] = F[v];
    return;
  }
  // conforming interior face (the list holds no other kind)
  const int L = fr.L, R = fr.R, dir = fr.face;
  int l1, l2, l3, r1, r2, r3;
  orders_of(m, L, l1, l2, l3);
  orders_of(m, R, r1, r2, r3);
  const int nL = l1 * l2 * l3, nR = r1 * r2 * r3;
  const int fL = 2 * dir + 1, fR = 2 * dir;
  const int la = dir == 0 ? l2 : l1, lb = dir == 2 ? l2 : l3, nf = la * lb;
#ifdef DG_BOUNDS_CHECK
  {
    const int ra = dir == 0 ? r2 : r1, rb = dir == 2 ? r2 : r3;
    if (fr.kind != 0 || ra != la || rb != lb || (unsigned)p >= (unsigned)nf) {
      flag_index(m);
      return;
    }
  }
#endif
  const int64_t oL = m.off[L], oR = m.off[R];
  double* outL = P.surf + 5 * (m.soff[L] + face_offset(l1, l2, l3, fL));
  double* outR = P.surf + 5 * (m.soff[R] + face_offset(r1, r2, r3, fR));
  const int a = p % la, b = p / la;
  const int iL = face_vidx(l1, l2, l3, fL, a, b), iR = face_vidx(r1, r2, r3, fR, a, b);
  double ja[3], nrm[3];
  face_metric<AFFINE>(m, L, nL, iL, dir, ja);
  const double area = unit_normal(ja, nrm);
  double qL[5], qR[5], F[5];
  for (int v = 0; v < 5; ++v) {
    qL[v] = P.q[5 * oL + v * nL + iL];
    qR[v] = P.q[5 * oR + v * nR + iR];
  }
  roe_face<AXIS>(gamma, dir, qL, qR, nrm, area, F);
  if (NS) {
    double gr[15], fa[3][5], fb[3][5];
    for (int v = 0; v < 5; ++v)
      for (int c = 0; c < 3; ++c) gr[v * 3 + c] = P.grad[15 * oL + (c * 5 + v) * nL + iL];
    viscous(m.ph, qL, gr, fa);
    for (int v = 0; v < 5; ++v)
      for (int c = 0; c < 3; ++c) gr[v * 3 + c] = P.grad[15 * oR + (c * 5 + v) * nR + iR];
    viscous(m.ph, qR, gr, fb);
    for (int v = 1; v < 5; ++v)
      F[v] -= 0.5 * ((fa[0][v] + fb[0][v]) * ja[0] + (fa[1][v] + fb[1][v]) * ja[1] + (fa[2][v] + fb[2][v]) * ja[2]);
  }
  for (int v = 0; v < 5; ++v) {
    outL[v * nf + p] = F[v];
    outR[v * nf + p] = F[v];
  }
}

// ------------------------------------------------------------ batched mortars
// p-nonconforming faces of affine Euler meshes, batched by shape signature
// (la, lb, ra, rb): the tangential node counts of the element behind the
// face (L) and ahead of it (R).  One CTA per batch; every phase runs flat over
// (face, point) of the batch, so the lanes stay busy whatever the shape:
//   gather both traces -> interpolate up to the mortar (Ma = max(la, ra),
//   Mb = max(lb, rb)) in two sum-factorised passes -> Roe at the mortar nodes
//   -> L2-project the flux back to each side in two passes -> store F*.
struct MortarBatch {
  int32_t first, count, la, lb, ra, rb;
};

struct MortarParams {
  MeshView m;
  const MortarBatch* batches;
  int n_batches;
  int n_mfaces;           // faces in the face list
  const int32_t* faces;   // [face][3]: L, R, dir
  const double* q;
  double* surf;
  const double* basis;
  const double* grad;     // general mortars, Navier-Stokes flux: the BR1 gradient
  const double* trace;    // affine Euler mortars: q's face traces (surf layout), or null to gather them from q
};

// shared memory (doubles) of one mortar batch
__host__ __device__ inline size_t mortar_batch_smem(const MortarBatch& B) {
  const int la = B.la, lb = B.lb, ra = B.ra, rb = B.rb;
  const int Ma = la > ra ? la : ra, Mb = lb > rb ? lb : rb;
  const int uL = (Ma * lb > la * Mb ? Ma * lb : la * Mb), uR = (Ma * rb > ra * Mb ? Ma * rb : ra * Mb);
  return (size_t)B.count * (5 * (la * lb + ra * rb + uL + uR + 2 * Ma * Mb) + 4);
}

// the tangential node counts (a, b) of element e's faces of direction dir
__device__ __forceinline__ void face_dims(const MeshView& m, int e, int dir, int& a, int& b) {
  const int n1 = m.ord[3 * e] + 1, n2 = m.ord[3 * e + 1] + 1, n3 = m.ord[3 * e + 2] + 1;
  a = dir == 0 ? n2 : n1;
  b = dir == 2 ? n2 : n3;
}

// A mortar batch of a block-uniform loop: its faces inside the face list,
// each face's elements in range with the batch's trace shapes, and the
// batch's shared memory (need, in doubles) inside the launch's allocation.
// In the checking build every thread of the block must call it.
__device__ __forceinline__ bool bad_batch(const MortarParams& P, const MortarBatch& B, size_t need) {
#ifdef DG_BOUNDS_CHECK
  const MeshView& m = P.m;
  bool bad = B.count < 1 || B.first < 0 || B.first > P.n_mfaces - B.count || B.la < 1 || B.lb < 1 || B.ra < 1 ||
             B.rb < 1 || B.la > DG_NP1 || B.lb > DG_NP1 || B.ra > DG_NP1 || B.rb > DG_NP1 ||
             need * sizeof(double) > dynamic_smem_bytes();
  for (int f = threadIdx.x; !bad && f < B.count; f += blockDim.x) {
    const int* fr = P.faces + 3 * (B.first + f);
    const int L = fr[0], R = fr[1], dir = fr[2];
    bad = (unsigned)L >= (unsigned)m.n_elem || (unsigned)R >= (unsigned)m.n_elem || (unsigned)dir >= 3u;
    if (!bad)
      bad = !elem_fits(m, L, m.ord[3 * L], m.ord[3 * L + 1], m.ord[3 * L + 2]) ||
            !elem_fits(m, R, m.ord[3 * R], m.ord[3 * R + 1], m.ord[3 * R + 2]);
    if (!bad) {
      int a, b;
      face_dims(m, L, dir, a, b);
      bad = a != B.la || b != B.lb;
      face_dims(m, R, dir, a, b);
      bad = bad || a != B.ra || b != B.rb;
    }
  }
  bad = __syncthreads_or(bad);
  if (bad && threadIdx.x == 0) flag_index(m);
  return bad;
#else
  (void)P;
  (void)B;
  (void)need;
  return false;
#endif
}

template <bool AXIS>
__global__ void __launch_bounds__(kVolThreads) mortar_kernel(MortarParams P) {
  extern __shared__ double smem[];
  const MeshView& m = P.m;
  const double gamma = m.ph.gamma;
  for (int it = blockIdx.x; it < P.n_batches; it += gridDim.x) {
    const MortarBatch B = P.batches[it];
    if (bad_batch(P, B, mortar_batch_smem(B))) continue;
    const int la = B.la, lb = B.lb, ra = B.ra, rb = B.rb, cnt = B.count;
    const int Ma = la > ra ? la : ra, Mb = lb > rb ? lb : rb;
    const int nfl = la * lb, nfr = ra * rb, nm = Ma * Mb;
    const bool upLa = la != Ma, upLb = lb != Mb, upRa = ra != Ma, upRb = rb != Mb;
    const int uL = (Ma * lb > la * Mb ? Ma * lb : la * Mb), uR = (Ma * rb > ra * Mb ? Ma * rb : ra * Mb);
    double* TL = smem;                       // [cnt][5][nfl] L trace
    double* TR = TL + cnt * 5 * nfl;         // [cnt][5][nfr] R trace
    double* UL = TR + cnt * 5 * nfr;         // [cnt][5][uL]  pass temporaries
    double* UR = UL + cnt * 5 * uL;          // [cnt][5][uR]
    double* QL = UR + cnt * 5 * uR;          // [cnt][5][nm]  mortar states, then the flux
    double* QR = QL + cnt * 5 * nm;          // [cnt][5][nm]
    double* NR = QR + cnt * 5 * nm;          // [cnt][4] unit normal, area
    // 1. gather traces, face normals
    for (int t = threadIdx.x; t < cnt * (nfl + nfr); t += blockDim.x) {
      const bool isL = t < cnt * nfl;
      const int tt = isL ? t : t - cnt * nfl;
      const int nf = isL ? nfl : nfr, na = isL ? la : ra;
      const int f = tt / nf, p = tt - f * nf;
      const int* fr = P.faces + 3 * (B.first + f);
      const int e = isL ? fr[0] : fr[1], dir = fr[2];
      int n1, n2, n3;
      orders_of(m, e, n1, n2, n3);
      double* T = (isL ? TL + f * 5 * nfl : TR + f * 5 * nfr) + p;
      if (P.trace) {   // the face's trace, contiguous [var][face node]
        const double* src = P.trace + 5 * (m.soff[e] + face_offset(n1, n2, n3, isL ? 2 * dir + 1 : 2 * dir)) + p;
        for (int v = 0; v < 5; ++v) T[v * nf] = src[v * nf];
      } else {
        const int n = n1 * n2 * n3;
        const int vi = face_vidx(n1, n2, n3, isL ? 2 * dir + 1 : 2 * dir, p % na, p / na);
        const int64_t o = m.off[e];
        for (int v = 0; v < 5; ++v) T[v * nf] = P.q[5 * o + v * n + vi];
      }
    }
    for (int f = threadIdx.x; f < cnt; f += blockDim.x) {
      const int* fr = P.faces + 3 * (B.first + f);
      double ja[3], nrm[3];
      for (int c = 0; c < 3; ++c) ja[c] = metric<true>(m.metric, fr[0], 0, 0, 0, 3 * fr[2] + c);
      const double area = unit_normal(ja, nrm);
      NR[4 * f + 0] = nrm[0];
      NR[4 * f + 1] = nrm[1];
      NR[4 * f + 2] = nrm[2];
      NR[4 * f + 3] = area;
    }
    __syncthreads();
    // 2. first interpolation pass (xi_a) for the sides that need it
    const double* IaL = P.basis + c_boff.I[la - 1][Ma - 1];
    const double* IaR = P.basis + c_boff.I[ra - 1][Ma - 1];
    {
      const int nL = upLa ? cnt * Ma * lb : 0, nR = upRa ? cnt * Ma * rb : 0;
      for (int t = threadIdx.x; t < nL + nR; t += blockDim.x) {
        const bool isL = t < nL;
        const int tt = isL ? t : t - nL;
        const int nb = isL ? lb : rb, na = isL ? la : ra, per = Ma * nb;
        const int f = tt / per, x = tt - f * per, m0 = x % Ma, b = x / Ma;
        const double* src = isL ? TL + f * 5 * nfl : TR + f * 5 * nfr;
        const double* Ia = isL ? IaL : IaR;
        double* dst = (isL ? UL + f * 5 * uL : UR + f * 5 * uR) + x;
        const int nsrc = na * nb;
        double acc[5] = {0, 0, 0, 0, 0};
        for (int a = 0; a < na; ++a) {
          const double w = __ldg(Ia + m0 * na + a);
          for (int v = 0; v < 5; ++v) acc[v] += w * src[v * nsrc + a + na * b];
        }
        for (int v = 0; v < 5; ++v) dst[v * per] = acc[v];
      }
    }
    __syncthreads();
    // 3. second interpolation pass (xi_b), or a copy, onto the mortar grid
    const double* IbL = P.basis + c_boff.I[lb - 1][Mb - 1];
    const double* IbR = P.basis + c_boff.I[rb - 1][Mb - 1];
    for (int t = threadIdx.x; t < 2 * cnt * nm; t += blockDim.x) {
      const bool isL = t < cnt * nm;
      const int tt = isL ? t : t - cnt * nm;
      const int f = tt / nm, x = tt - f * nm, m0 = x % Ma, m1 = x / Ma;
      const bool upa = isL ? upLa : upRa, upb = isL ? upLb : upRb;
      const int nb = isL ? lb : rb;
      // source grid (Ma x nb): the pass-a result, or the trace itself
      const double* src = upa ? (isL ? UL + f * 5 * uL : UR + f * 5 * uR) : (isL ? TL + f * 5 * nfl : TR + f * 5 * nfr);
      const int nsrc = Ma * nb;
      double* dst = (isL ? QL : QR) + f * 5 * nm + x;
      if (upb) {
        const double* Ib = isL ? IbL : IbR;
        double acc[5] = {0, 0, 0, 0, 0};
        for (int b = 0; b < nb; ++b) {
          const double w = __ldg(Ib + m1 * nb + b);
          for (int v = 0; v < 5; ++v) acc[v] += w * src[v * nsrc + m0 + Ma * b];
        }
        for (int v = 0; v < 5; ++v) dst[v * nm] = acc[v];
      } else {
        for (int v = 0; v < 5; ++v) dst[v * nm] = src[v * nsrc + m0 + Ma * m1];
      }
    }
    __syncthreads();
    // 4. Roe at the mortar nodes (flux scaled by the face area, stored in QL)
    for (int t = threadIdx.x; t < cnt * nm; t += blockDim.x) {
      const int f = t / nm, x = t - f * nm;
      double qa[5], qb[5], F[5];
      for (int v = 0; v < 5; ++v) {
        qa[v] = QL[f * 5 * nm + v * nm + x];
        qb[v] = QR[f * 5 * nm + v * nm + x];
      }
      const double nrm[3] = {NR[4 * f], NR[4 * f + 1], NR[4 * f + 2]};
      roe_face<AXIS>(gamma, P.faces[3 * (B.first + f) + 2], qa, qb, nrm, NR[4 * f + 3], F);
      for (int v = 0; v < 5; ++v) QL[f * 5 * nm + v * nm + x] = F[v];
    }
    __syncthreads();
    // 5. first projection pass (xi_a) back to each side that needs it
    const double* PaL = P.basis + c_boff.P[Ma - 1][la - 1];
    const double* PaR = P.basis + c_boff.P[Ma - 1][ra - 1];
    {
      const int nL = upLa ? cnt * la * Mb : 0, nR = upRa ? cnt * ra * Mb : 0;
      for (int t = threadIdx.x; t < nL + nR; t += blockDim.x) {
        const bool isL = t < nL;
        const int tt = isL ? t : t - nL;
        const int na = isL ? la : ra, per = na * Mb;
        const int f = tt / per, x = tt - f * per, a = x % na, m1 = x / na;
        const double* Pa = isL ? PaL : PaR;
        const double* src = QL + f * 5 * nm;
        double* dst = (isL ? UL + f * 5 * uL : UR + f * 5 * uR) + x;
        double acc[5] = {0, 0, 0, 0, 0};
        for (int m0 = 0; m0 < Ma; ++m0) {
          const double w = __ldg(Pa + a * Ma + m0);
          for (int v = 0; v < 5; ++v) acc[v] += w * src[v * nm + m0 + Ma * m1];
        }
        for (int v = 0; v < 5; ++v) dst[v * per] = acc[v];
      }
    }
    __syncthreads();
    // 6. second projection pass (xi_b), or a copy, onto each side's face grid
    const double* PbL = P.basis + c_boff.P[Mb - 1][lb - 1];
    const double* PbR = P.basis + c_boff.P[Mb - 1][rb - 1];
    for (int t = threadIdx.x; t < cnt * (nfl + nfr); t += blockDim.x) {
      const bool isL = t < cnt * nfl;
      const int tt = isL ? t : t - cnt * nfl;
      const int nf = isL ? nfl : nfr, na = isL ? la : ra;
      const int f = tt / nf, x = tt - f * nf, a = x % na, b = x / na;
      const bool upa = isL ? upLa : upRa, upb = isL ? upLb : upRb;
      // source grid (na x Mb): the pass-5 result, or the mortar flux itself
      const double* src = upa ? (isL ? UL + f * 5 * uL : UR + f * 5 * uR) : QL + f * 5 * nm;
      const int nsrc = na * Mb;
      double out[5];
      if (upb) {
        const double* Pb = isL ? PbL : PbR;
        for (int v = 0; v < 5; ++v) out[v] = 0.0;
        for (int m1 = 0; m1 < Mb; ++m1) {
          const double w = __ldg(Pb + b * Mb + m1);
          for (int v = 0; v < 5; ++v) out[v] += w * src[v * nsrc + a + na * m1];
        }
      } else {
        for (int v = 0; v < 5; ++v) out[v] = src[v * nsrc + a + na * b];
      }
      const int* fr = P.faces + 3 * (B.first + f);
      const int e = isL ? fr[0] : fr[1], dir = fr[2];
      int n1, n2, n3;
      orders_of(m, e, n1, n2, n3);
      double* dst = P.surf + 5 * (m.soff[e] + face_offset(n1, n2, n3, isL ? 2 * dir + 1 : 2 * dir)) + x;
      for (int v = 0; v < 5; ++v) dst[v * nf] = out[v];
    }
    __syncthreads();
  }
}

// ------------------------------------------------- general (curved, NS) mortars
// p-nonconforming faces of curved or Navier-Stokes meshes, in the same shape
// batches.  The two sides' J a^dir at a curved nonconforming face differ (each
// element's metric comes from the geometry at its own order), so each side
// takes the flux with its own normal, as a conforming face would, from both
// traces on the mortar grid:
//   gather each side's trace (q; the BR1 gradient for the Navier-Stokes flux)
//   and its own J a^dir -> interpolate up to the mortar in two passes ->
//   per side F* = |J a| Roe(q-, q+, n_side) - {{f_v}} . J a_side (BR1 average),
//   or for the BR1 gradient pass S = {{q}} J a_side -> L2-project each side's
//   output back to its own face grid in two passes -> store.
// MODE 0: Euler flux, 1: Navier-Stokes flux, 2: BR1 q-hat (J a) into surfq.
template <int MODE>
struct GMortar {
  static constexpr int nq = MODE == 1 ? 20 : 5;   // q and, for the NS flux, its gradient [v*3+c]
  static constexpr int nin = nq + 3;              // ... and the side's own J a^dir
  static constexpr int nout = MODE == 2 ? 15 : 5;
  static constexpr int nmid = nin > nout ? nin : nout;
};

template <int MODE>
__host__ __device__ inline size_t mortar_general_smem(const MortarBatch& B) {
  const int la = B.la, lb = B.lb, ra = B.ra, rb = B.rb;
  const int Ma = la > ra ? la : ra, Mb = lb > rb ? lb : rb, nm = Ma * Mb;
  const int uL = (Ma * lb > la * Mb ? Ma * lb : la * Mb), uR = (Ma * rb > ra * Mb ? Ma * rb : ra * Mb);
  return (size_t)B.count * ((size_t)GMortar<MODE>::nin * (la * lb + ra * rb + 2 * nm) +
                            (size_t)GMortar<MODE>::nmid * (uL + uR) + 2 * (size_t)GMortar<MODE>::nout * nm);
}

// Two CTAs a SM (batches hold at most 96 KB of shared memory): the
// Navier-Stokes flux mode then fits 128 registers with a few spilled values,
// where it took 152 and one CTA; 6% faster RK steps on a cylinder of random
// orders 1-6.
template <bool AFFINE, int MODE>
__global__ void __launch_bounds__(kVolThreads, 2) mortar_general_kernel(MortarParams P) {
  typedef GMortar<MODE> G;
  constexpr int NIN = G::nin, NQ = G::nq, NOUT = G::nout, NMID = G::nmid;
  extern __shared__ double smem[];
  const MeshView& m = P.m;
  const double gamma = m.ph.gamma;
  for (int it = blockIdx.x; it < P.n_batches; it += gridDim.x) {
    const MortarBatch B = P.batches[it];
    if (bad_batch(P, B, mortar_general_smem<MODE>(B))) continue;
    const int la = B.la, lb = B.lb, ra = B.ra, rb = B.rb, cnt = B.count;
    const int Ma = la > ra ? la : ra, Mb = lb > rb ? lb : rb;
    const int nfl = la * lb, nfr = ra * rb, nm = Ma * Mb;
    const bool upLa = la != Ma, upLb = lb != Mb, upRa = ra != Ma, upRb = rb != Mb;
    const int uL = (Ma * lb > la * Mb ? Ma * lb : la * Mb), uR = (Ma * rb > ra * Mb ? Ma * rb : ra * Mb);
    double* TL = smem;                          // [cnt][NIN][nfl] L trace and J a
    double* TR = TL + cnt * NIN * nfl;          // [cnt][NIN][nfr]
    double* UL = TR + cnt * NIN * nfr;          // [cnt][NMID][uL] pass temporaries
    double* UR = UL + cnt * NMID * uL;          // [cnt][NMID][uR]
    double* QL = UR + cnt * NMID * uR;          // [cnt][NIN][nm] on the mortar grid
    double* QR = QL + cnt * NIN * nm;           // [cnt][NIN][nm]
    double* OL = QR + cnt * NIN * nm;           // [cnt][NOUT][nm] each side's output
    double* OR = OL + cnt * NOUT * nm;          // [cnt][NOUT][nm]
    // 1. gather both traces and each side's own J a^dir
    for (int t = threadIdx.x; t < cnt * (nfl + nfr); t += blockDim.x) {
      const bool isL = t < cnt * nfl;
      const int tt = isL ? t : t - cnt * nfl;
      const int nf = isL ? nfl : nfr, na = isL ? la : ra;
      const int f = tt / nf, p = tt - f * nf;
      const int* fr = P.faces + 3 * (B.first + f);
      const int e = isL ? fr[0] : fr[1], dir = fr[2];
      int n1, n2, n3;
      orders_of(m, e, n1, n2, n3);
      const int n = n1 * n2 * n3;
      const int vi = face_vidx(n1, n2, n3, isL ? 2 * dir + 1 : 2 * dir, p % na, p / na);
      const int64_t o = m.off[e];
      double* T = (isL ? TL + f * NIN * nfl : TR + f * NIN * nfr) + p;
      for (int v = 0; v < 5; ++v) T[v * nf] = P.q[5 * o + v * n + vi];
      if (MODE == 1)
        for (int v = 0; v < 5; ++v)
          for (int c = 0; c < 3; ++c) T[(5 + v * 3 + c) * nf] = P.grad[15 * o + (c * 5 + v) * n + vi];
      double ja[3];
      face_metric<AFFINE>(m, e, n, vi, dir, ja);
      for (int c = 0; c < 3; ++c) T[(NQ + c) * nf] = ja[c];
    }
    __syncthreads();
    // 2. first interpolation pass (xi_a) for the sides that need it
    const double* IaL = P.basis + c_boff.I[la - 1][Ma - 1];
    const double* IaR = P.basis + c_boff.I[ra - 1][Ma - 1];
    {
      const int nL = upLa ? cnt * Ma * lb : 0, nR = upRa ? cnt * Ma * rb : 0;
      for (int t = threadIdx.x; t < nL + nR; t += blockDim.x) {
        const bool isL = t < nL;
        const int tt = isL ? t : t - nL;
        const int nb = isL ? lb : rb, na = isL ? la : ra, per = Ma * nb;
        const int f = tt / per, x = tt - f * per, m0 = x % Ma, b = x / Ma;
        const double* src = isL ? TL + f * NIN * nfl : TR + f * NIN * nfr;
        const double* Ia = isL ? IaL : IaR;
        double* dst = (isL ? UL + f * NMID * uL : UR + f * NMID * uR) + x;
        const int nsrc = na * nb;
        double acc[NIN];
        for (int c = 0; c < NIN; ++c) acc[c] = 0.0;
        for (int a = 0; a < na; ++a) {
          const double w = __ldg(Ia + m0 * na + a);
          for (int c = 0; c < NIN; ++c) acc[c] += w * src[c * nsrc + a + na * b];
        }
        for (int c = 0; c < NIN; ++c) dst[c * per] = acc[c];
      }
    }
    __syncthreads();
    // 3. second interpolation pass (xi_b), or a copy, onto the mortar grid
    const double* IbL = P.basis + c_boff.I[lb - 1][Mb - 1];
    const double* IbR = P.basis + c_boff.I[rb - 1][Mb - 1];
    for (int t = threadIdx.x; t < 2 * cnt * nm; t += blockDim.x) {
      const bool isL = t < cnt * nm;
      const int tt = isL ? t : t - cnt * nm;
      const int f = tt / nm, x = tt - f * nm, m0 = x % Ma, m1 = x / Ma;
      const bool upa = isL ? upLa : upRa, upb = isL ? upLb : upRb;
      const int nb = isL ? lb : rb;
      const double* src = upa ? (isL ? UL + f * NMID * uL : UR + f * NMID * uR)
                              : (isL ? TL + f * NIN * nfl : TR + f * NIN * nfr);
      const int nsrc = Ma * nb;
      double* dst = (isL ? QL : QR) + f * NIN * nm + x;
      if (upb) {
        const double* Ib = isL ? IbL : IbR;
        double acc[NIN];
        for (int c = 0; c < NIN; ++c) acc[c] = 0.0;
        for (int b = 0; b < nb; ++b) {
          const double w = __ldg(Ib + m1 * nb + b);
          for (int c = 0; c < NIN; ++c) acc[c] += w * src[c * nsrc + m0 + Ma * b];
        }
        for (int c = 0; c < NIN; ++c) dst[c * nm] = acc[c];
      } else {
        for (int c = 0; c < NIN; ++c) dst[c * nm] = src[c * nsrc + m0 + Ma * m1];
      }
    }
    __syncthreads();
    // 4. each side's output at the mortar nodes, with its own J a^dir
    for (int t = threadIdx.x; t < cnt * nm; t += blockDim.x) {
      const int f = t / nm, x = t - f * nm;
      const double* ql = QL + f * NIN * nm + x;
      const double* qr = QR + f * NIN * nm + x;
      double qa[5], qb[5], jl[3], jr[3];
      for (int v = 0; v < 5; ++v) {
        qa[v] = ql[v * nm];
        qb[v] = qr[v * nm];
      }
      for (int c = 0; c < 3; ++c) {
        jl[c] = ql[(NQ + c) * nm];
        jr[c] = qr[(NQ + c) * nm];
      }
      double* ol = OL + f * NOUT * nm + x;
      double* orr = OR + f * NOUT * nm + x;
      if (MODE == 2) {
        for (int v = 0; v < 5; ++v) {
          const double qh = 0.5 * (qa[v] + qb[v]);
          for (int c = 0; c < 3; ++c) {
            ol[(v * 3 + c) * nm] = qh * jl[c];
            orr[(v * 3 + c) * nm] = qh * jr[c];
          }
        }
        continue;
      }
      double nl[3], nr[3], FLv[5], FRv[5];
      const double al = unit_normal(jl, nl), ar = unit_normal(jr, nr);
      roe_face<false>(gamma, 0, qa, qb, nl, al, FLv);
      roe_face<false>(gamma, 0, qa, qb, nr, ar, FRv);
      if (MODE == 1) {
        double g[15], fa[3][5], fb[3][5];
        for (int c = 0; c < 15; ++c) g[c] = ql[(5 + c) * nm];
        viscous(m.ph, qa, g, fa);
        for (int c = 0; c < 15; ++c) g[c] = qr[(5 + c) * nm];
        viscous(m.ph, qb, g, fb);
        for (int v = 1; v < 5; ++v) {
          const double s0 = fa[0][v] + fb[0][v], s1 = fa[1][v] + fb[1][v], s2 = fa[2][v] + fb[2][v];
          FLv[v] -= 0.5 * (s0 * jl[0] + s1 * jl[1] + s2 * jl[2]);
          FRv[v] -= 0.5 * (s0 * jr[0] + s1 * jr[1] + s2 * jr[2]);
        }
      }
      for (int v = 0; v < 5; ++v) {
        ol[v * nm] = FLv[v];
        orr[v * nm] = FRv[v];
      }
    }
    __syncthreads();
    // 5. first projection pass (xi_a) back to each side that needs it
    const double* PaL = P.basis + c_boff.P[Ma - 1][la - 1];
    const double* PaR = P.basis + c_boff.P[Ma - 1][ra - 1];
    {
      const int nL = upLa ? cnt * la * Mb : 0, nR = upRa ? cnt * ra * Mb : 0;
      for (int t = threadIdx.x; t < nL + nR; t += blockDim.x) {
        const bool isL = t < nL;
        const int tt = isL ? t : t - nL;
        const int na = isL ? la : ra, per = na * Mb;
        const int f = tt / per, x = tt - f * per, a = x % na, m1 = x / na;
        const double* Pa = isL ? PaL : PaR;
        const double* src = (isL ? OL : OR) + f * NOUT * nm;
        double* dst = (isL ? UL + f * NMID * uL : UR + f * NMID * uR) + x;
        double acc[NOUT];
        for (int c = 0; c < NOUT; ++c) acc[c] = 0.0;
        for (int m0 = 0; m0 < Ma; ++m0) {
          const double w = __ldg(Pa + a * Ma + m0);
          for (int c = 0; c < NOUT; ++c) acc[c] += w * src[c * nm + m0 + Ma * m1];
        }
        for (int c = 0; c < NOUT; ++c) dst[c * per] = acc[c];
      }
    }
    __syncthreads();
    // 6. second projection pass (xi_b), or a copy, onto each side's face grid; store
    const double* PbL = P.basis + c_boff.P[Mb - 1][lb - 1];
    const double* PbR = P.basis + c_boff.P[Mb - 1][rb - 1];
    for (int t = threadIdx.x; t < cnt * (nfl + nfr); t += blockDim.x) {
      const bool isL = t < cnt * nfl;
      const int tt = isL ? t : t - cnt * nfl;
      const int nf = isL ? nfl : nfr, na = isL ? la : ra;
      const int f = tt / nf, x = tt - f * nf, a = x % na, b = x / na;
      const bool upa = isL ? upLa : upRa, upb = isL ? upLb : upRb;
      const double* src = upa ? (isL ? UL + f * NMID * uL : UR + f * NMID * uR) : (isL ? OL : OR) + f * NOUT * nm;
      const int nsrc = na * Mb;
      double out[NOUT];
      if (upb) {
        const double* Pb = isL ? PbL : PbR;
        for (int c = 0; c < NOUT; ++c) out[c] = 0.0;
        for (int m1 = 0; m1 < Mb; ++m1) {
          const double w = __ldg(Pb + b * Mb + m1);
          for (int c = 0; c < NOUT; ++c) out[c] += w * src[c * nsrc + a + na * m1];
        }
      } else {
        for (int c = 0; c < NOUT; ++c) out[c] = src[c * nsrc + a + na * b];
      }
      const int* fr = P.faces + 3 * (B.first + f);
      const int e = isL ? fr[0] : fr[1], dir = fr[2];
      int n1, n2, n3;
      orders_of(m, e, n1, n2, n3);
      double* dst = (MODE == 2 ? P.surf + 15 * (m.soff[e] + face_offset(n1, n2, n3, isL ? 2 * dir + 1 : 2 * dir))
                               : P.surf + 5 * (m.soff[e] + face_offset(n1, n2, n3, isL ? 2 * dir + 1 : 2 * dir)));
      for (int c = 0; c < NOUT; ++c) dst[c * nf + x] = out[c];
    }
    __syncthreads();
  }
}


// BR1 trace q-hat (J a^dir) on every face; conforming faces only.
template <bool AFFINE>
__global__ void __launch_bounds__(32 * kFaceWarps) face_qhat_kernel(FaceParams P, double* surfq) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int fidx = blockIdx.x * kFaceWarps + warp;
  if (fidx >= P.n_faces) return;
  const FaceRec fr = P.faces[fidx];
  if (bad_face(P.m, fr)) return;
  const MeshView& m = P.m;
  if (fr.kind == 2) {
    int e = fr.L, f = fr.face, tag = fr.R, dir = f >> 1;
    int n1, n2, n3;
    orders_of(m, e, n1, n2, n3);
    int n = n1 * n2 * n3;
    int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3, nf = na * nb;
    int64_t o = m.off[e];
    double* out = surfq + 15 * (m.soff[e] + face_offset(n1, n2, n3, f));
    for (int p = lane; p < nf; p += 32) {
      int vi = face_vidx(n1, n2, n3, f, p % na, p / na);
      double qi[5], qh[5], ja[3];
      for (int v = 0; v < 5; ++v) qi[v] = P.q[5 * o + v * n + vi];
      face_metric<AFFINE>(m, e, n, vi, dir, ja);
      bc_qhat(m.ph, tag, qi, qh);
      for (int v = 0; v < 5; ++v)
        for (int c = 0; c < 3; ++c) out[(v * 3 + c) * nf + p] = qh[v] * ja[c];
    }
    return;
  }
  const int L = fr.L, R = fr.R, dir = fr.face;
  int l1, l2, l3, r1, r2, r3;
  orders_of(m, L, l1, l2, l3);
  orders_of(m, R, r1, r2, r3);
  const int nL = l1 * l2 * l3, nR = r1 * r2 * r3;
  const int64_t oL = m.off[L], oR = m.off[R];
  const int la = dir == 0 ? l2 : l1, lb = dir == 2 ? l2 : l3, nf = la * lb;
  double* outL = surfq + 15 * (m.soff[L] + face_offset(l1, l2, l3, 2 * dir + 1));
  double* outR = surfq + 15 * (m.soff[R] + face_offset(r1, r2, r3, 2 * dir));
  for (int p = lane; p < nf; p += 32) {
    int a = p % la, b = p / la;
    int iL = face_vidx(l1, l2, l3, 2 * dir + 1, a, b), iR = face_vidx(r1, r2, r3, 2 * dir, a, b);
    double ja[3];
    face_metric<AFFINE>(m, L, nL, iL, dir, ja);
    for (int v = 0; v < 5; ++v) {
      double qh = 0.5 * (P.q[5 * oL + v * nL + iL] + P.q[5 * oR + v * nR + iR]);
      for (int c = 0; c < 3; ++c) {
        outL[(v * 3 + c) * nf + p] = qh * ja[c];
        outR[(v * 3 + c) * nf + p] = qh * ja[c];
      }
    }
  }
}

// ------------------------------------------------------ volume-type kernels
// the gas constants of the CFL time scale in precision T
template <typename T>
struct ScaleConst {
  T gm1, gamma, mu, gpr;   // gamma - 1, gamma, mu, max(1, gamma/Pr)
  int ns;                  // Navier-Stokes
};

struct VolParams {
  MeshView m;
  const WorkItem* items;
  int n_items;              // number of work items to run (entries of ilist, or all items)
  const int32_t* ilist;     // items of this launch (one shared-memory size class), or null for all
  const int32_t* elist;
  const double* q;
  const double* grad;
  const double* surf;
  const double* surfq;
  const double* basis;
  double* out;        // residual or gradient
  double* q_io;       // RK: state updated in place
  double* g_io;       // RK: register
  double* trace_out;  // RK, affine Euler: the updated state at every element face node (surf layout), or null
  const double* dt;
  double rkA, rkB;
  int rk;             // 0: write residual; 1: RK stage
  int rk_first;       // first stage: G = dt R (A = 0)
  int isolated;
  unsigned* err;
  // CFL reduction: the gas constants in both precisions (formed on the host)
  // and the FP32 copy of the affine metric
  ScaleConst<float> k32;
  ScaleConst<double> k64;
  const float* metric32;
  int n_items_all;    // length of items (the bound of an ilist entry)
};

// Sum-factorised GL derivative of a [3][nv][n] contravariant-flux tile at
// node (i,j,k): out[v] = sum_m D1[i][m] F1[v][m,j,k] + D2[j][m] F2[v][i,m,k] + D3[k][m] F3[v][i,j,m]
template <int NVAR>
__device__ __forceinline__ void div_tile(const double* __restrict__ F, int n1, int n2, int n3, int i, int j, int k,
                                         const double* D1, const double* D2, const double* D3, double out[NVAR]) {
  const int n = n1 * n2 * n3;
  for (int v = 0; v < NVAR; ++v) out[v] = 0.0;
  const double* F1 = F;
  const double* F2 = F + NVAR * n;
  const double* F3 = F + 2 * NVAR * n;
  int base1 = n1 * (j + n2 * k);
  for (int mm = 0; mm < n1; ++mm) {
    double d = __ldg(D1 + i * n1 + mm);
    for (int v = 0; v < NVAR; ++v) out[v] += d * F1[v * n + base1 + mm];
  }
  int base2 = i + n1 * n2 * k;
  for (int mm = 0; mm < n2; ++mm) {
    double d = __ldg(D2 + j * n2 + mm);
    for (int v = 0; v < NVAR; ++v) out[v] += d * F2[v * n + base2 + n1 * mm];
  }
  int base3 = i + n1 * j;
  for (int mm = 0; mm < n3; ++mm) {
    double d = __ldg(D3 + k * n3 + mm);
    for (int v = 0; v < NVAR; ++v) out[v] += d * F3[v * n + base3 + n1 * n2 * mm];
  }
}

// The off-diagonal part of div_tile: the GL derivative matrix has a zero
// diagonal at interior nodes and D_00 = -D_NN = -N(N+1)/4 at the end nodes,
// which the volume kernel applies with the surface lift (it multiplies the
// same end-node flux).  Each node runs the n-1 taps m != i in the rotated
// order i+1, ..., n-1, 0, ..., i-1, so the lanes of a warp (consecutive i)
// issue the same number of FP64 instructions: one DFMA per variable and tap
// fewer than with the diagonal, n-1 instead of n.
template <int NVAR>
__device__ __forceinline__ void div_tile_offdiag(const double* __restrict__ F, int n1, int n2, int n3, int i, int j,
                                                 int k, const double* D1, const double* D2, const double* D3,
                                                 double out[NVAR]) {
  const int n = n1 * n2 * n3;
  for (int v = 0; v < NVAR; ++v) out[v] = 0.0;
  const double* F1 = F + n1 * (j + n2 * k);
  const double* F2 = F + NVAR * n + i + n1 * n2 * k;
  const double* F3 = F + 2 * NVAR * n + i + n1 * j;
  for (int t = 1, mm = i; t < n1; ++t) {
    mm = mm + 1 == n1 ? 0 : mm + 1;
    const double d = __ldg(D1 + i * n1 + mm);
    for (int v = 0; v < NVAR; ++v) out[v] += d * F1[v * n + mm];
  }
  for (int t = 1, mm = j; t < n2; ++t) {
    mm = mm + 1 == n2 ? 0 : mm + 1;
    const double d = __ldg(D2 + j * n2 + mm);
    for (int v = 0; v < NVAR; ++v) out[v] += d * F2[v * n + n1 * mm];
  }
  for (int t = 1, mm = k; t < n3; ++t) {
    mm = mm + 1 == n3 ? 0 : mm + 1;
    const double d = __ldg(D3 + k * n3 + mm);
    for (int v = 0; v < NVAR; ++v) out[v] += d * F3[v * n + n1 * n2 * mm];
  }
}

// Volume residual of one work item per iteration (a tile of same-order
// elements), in four shared-memory phases:
//  1. per node: primitive variables, contravariant fluxes Ft^i = J a^i . f
//     (AXIS: J a^i = (J a^i_i) e_i, so Ft^i = J a^i_i f_i);
//  2. per node: the off-diagonal part of the sum-factorised GL derivative
//     sum_i D^(i) Ft^i -> V (div_tile_offdiag);
//  3. per face node, one direction at a time (the two faces of a direction
//     touch disjoint nodes): the surface lift +-(F* - Ft^dir)/w_end and the
//     derivative's end-node diagonal D_ee Ft^dir = -+Ft^dir/(2 w_end)
//     together, V += +-(F* / w_end - Ft^dir / (2 w_end)), with every lane
//     busy; the isolated residual (F* = Ft) keeps the diagonal alone;
//  4. per node: R = -V/J, written or fused into the RK3 stage.
template <bool AFFINE, bool AXIS, bool NS, int THREADS>
__global__ void __launch_bounds__(THREADS) volume_kernel(VolParams P) {
  extern __shared__ double smem[];
  const MeshView& m = P.m;
  const double gm1 = m.ph.gamma - 1.0;
  for (int it = blockIdx.x; it < P.n_items; it += gridDim.x) {
    WorkItem w;
    if (!take_item(P.m, P.items, P.ilist ? P.ilist[it] : it, P.n_items_all, P.elist, 20, w)) continue;
    const int n1 = w.n1 + 1, n2 = w.n2 + 1, n3 = w.n3 + 1, n = n1 * n2 * n3;
    const int slots = w.count * n;
    double* Ft = smem;                                // [count][3][5][n]
    double* V = smem + (size_t)w.count * 15 * n;      // [count][5][n]
    // phase 1
    for (int s = threadIdx.x; s < slots; s += blockDim.x) {
      const int el = s / n, p = s - el * n;
      const int e = P.elist[w.first + el];
      const int64_t o = m.off[e];
      double q[5];
      for (int v = 0; v < 5; ++v) q[v] = P.q[5 * o + v * n + p];
      const double ir = 1.0 / q[0];
      const double u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
      const double pr = gm1 * (q[4] - 0.5 * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
      if (!(q[0] > 0.0) || !(pr > 0.0)) atomicOr(P.err, 1u);
      double* F = Ft + (size_t)el * 15 * n;
      if (AXIS && !NS) {
        const double Epr = q[4] + pr;
        for (int i = 0; i < 3; ++i) {
          const double a = metric<true>(m.metric, e, 0, n, p, 4 * i);   // J a^i_i
          const double uc = a * u[i];                                     // contravariant velocity
          F[(i * 5 + 0) * n + p] = q[0] * uc;
          F[(i * 5 + 1) * n + p] = q[1] * uc;
          F[(i * 5 + 2) * n + p] = q[2] * uc;
          F[(i * 5 + 3) * n + p] = q[3] * uc;
          F[(i * 5 + 1 + i) * n + p] += a * pr;
          F[(i * 5 + 4) * n + p] = uc * Epr;
        }
      } else {
        double f[3][5];
        for (int d = 0; d < 3; ++d) {
          f[d][0] = q[1 + d];
          f[d][1] = q[1] * u[d];
          f[d][2] = q[2] * u[d];
          f[d][3] = q[3] * u[d];
          f[d][1 + d] += pr;
          f[d][4] = u[d] * (q[4] + pr);
        }
        if (NS) {
          double g[15], fv[3][5];
          for (int v = 0; v < 5; ++v)
            for (int c = 0; c < 3; ++c) g[v * 3 + c] = P.grad[15 * o + (c * 5 + v) * n + p];
          viscous(m.ph, q, g, fv);
          for (int d = 0; d < 3; ++d)
            for (int v = 0; v < 5; ++v) f[d][v] -= fv[d][v];
        }
        for (int i = 0; i < 3; ++i) {
          const double ja0 = metric<AFFINE>(m.metric, e, o, n, p, 3 * i + 0);
          const double ja1 = metric<AFFINE>(m.metric, e, o, n, p, 3 * i + 1);
          const double ja2 = metric<AFFINE>(m.metric, e, o, n, p, 3 * i + 2);
          for (int v = 0; v < 5; ++v) F[(i * 5 + v) * n + p] = ja0 * f[0][v] + ja1 * f[1][v] + ja2 * f[2][v];
        }
      }
    }
    __syncthreads();
    // phase 2
    const double* D1 = P.basis + c_boff.D[w.n1];
    const double* D2 = P.basis + c_boff.D[w.n2];
    const double* D3 = P.basis + c_boff.D[w.n3];
    for (int s = threadIdx.x; s < slots; s += blockDim.x) {
      const int el = s / n, p = s - el * n;
      const int i = p % n1, j = (p / n1) % n2, k = p / (n1 * n2);
      double vol[5];
      div_tile_offdiag<5>(Ft + (size_t)el * 15 * n, n1, n2, n3, i, j, k, D1, D2, D3, vol);
      double* Vv = V + (size_t)el * 5 * n;
      for (int v = 0; v < 5; ++v) Vv[v * n + p] = vol[v];
    }
    __syncthreads();
    // phase 3
    for (int dir = 0; dir < 3; ++dir) {
      const int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3, fsz = na * nb;
      const int Nd = dir == 0 ? w.n1 : (dir == 1 ? w.n2 : w.n3);
      const double inv_w = 0.5 * Nd * (Nd + 1);   // 1 / w_0 = 1 / w_N = N(N+1)/2
      const int per_el = 2 * fsz;
      for (int s = threadIdx.x; s < w.count * per_el; s += blockDim.x) {
        const int el = s / per_el, r = s - el * per_el;
        const int side = r / fsz, fn = r - side * fsz;
        const int f = 2 * dir + side;
        const int p = face_vidx(n1, n2, n3, f, fn % na, fn / na);
        const double* F = Ft + (size_t)el * 15 * n + dir * 5 * n + p;
        double* Vv = V + (size_t)el * 5 * n + p;
        const double sg = side ? inv_w : -inv_w;     // the lift's sign and 1 / w_end
        if (P.isolated) {
          for (int v = 0; v < 5; ++v) Vv[v * n] += (0.5 * sg) * F[v * n];   // D_ee Ft^dir
        } else {
          const int e = P.elist[w.first + el];
          const double* Fs = P.surf + 5 * (m.soff[e] + face_offset(n1, n2, n3, f)) + fn;
          for (int v = 0; v < 5; ++v) Vv[v * n] += sg * Fs[v * fsz] - (0.5 * sg) * F[v * n];
        }
      }
      __syncthreads();
    }
    // phase 4
    for (int s = threadIdx.x; s < slots; s += blockDim.x) {
      const int el = s / n, p = s - el * n;
      const int e = P.elist[w.first + el];
      const int64_t o = m.off[e];
      const double miJ = -metric<AFFINE>(m.metric, e, o, n, p, 10);
      double* Vv = V + (size_t)el * 5 * n + p;
      if (P.rk) {
        const double c = *P.dt * miJ;   // dt R = (-dt/J) V
        double qn[5];
        for (int v = 0; v < 5; ++v) {
          const int64_t idx = 5 * o + v * n + p;
          const double dr = c * Vv[v * n];
          const double g = P.rk_first ? dr : P.rkA * P.g_io[idx] + dr;
          P.g_io[idx] = g;
          qn[v] = P.q_io[idx] + P.rkB * g;
          P.q_io[idx] = qn[v];
        }
        if (P.trace_out)   // the new state replaces V (read by this thread only) for phase 5
          for (int v = 0; v < 5; ++v) Vv[v * n] = qn[v];
      } else {
        for (int v = 0; v < 5; ++v) P.out[5 * o + v * n + p] = Vv[v * n] * miJ;
      }
    }
    __syncthreads();
    // phase 5 (RK, affine Euler): the new state at every element face node into
    // the trace buffer, contiguous per face as the next stage's mortars read it
    if (P.rk && P.trace_out) {
      const int fs[3] = {n2 * n3, n1 * n3, n1 * n2};
      const int per_el = 2 * (fs[0] + fs[1] + fs[2]);
      for (int s = threadIdx.x; s < w.count * per_el; s += blockDim.x) {
        const int el = s / per_el;
        int r = s - el * per_el, f = 0;
        while (r >= fs[f >> 1]) r -= fs[f++ >> 1];
        const int na = f < 2 ? n2 : n1;
        const int p = face_vidx(n1, n2, n3, f, r % na, r / na);
        const int e = P.elist[w.first + el];
        const double* Vv = V + (size_t)el * 5 * n + p;
        double* t = P.trace_out + 5 * (m.soff[e] + face_offset(n1, n2, n3, f)) + r;
        for (int v = 0; v < 5; ++v) t[v * fs[f >> 1]] = Vv[v * n];
      }
      __syncthreads();
    }
  }
}

// BR1 gradient (strong form): J g_c = sum_i D^(i)(J a^i_c q) + lifted (q-hat - q) J a^dir_c.
template <bool AFFINE>
__global__ void __launch_bounds__(kVolThreads) gradient_kernel(VolParams P) {
  extern __shared__ double smem[];
  const MeshView& m = P.m;
  for (int it = blockIdx.x; it < P.n_items; it += gridDim.x) {
    WorkItem w;
    if (!take_item(P.m, P.items, P.ilist ? P.ilist[it] : it, P.n_items_all, P.elist, 15, w)) continue;
    const int n1 = w.n1 + 1, n2 = w.n2 + 1, n3 = w.n3 + 1, n = n1 * n2 * n3;
    const int slots = w.count * n;
    const double* D1 = P.basis + c_boff.D[w.n1];
    const double* D2 = P.basis + c_boff.D[w.n2];
    const double* D3 = P.basis + c_boff.D[w.n3];
    for (int c = 0; c < 3; ++c) {
      for (int s = threadIdx.x; s < slots; s += blockDim.x) {
        const int el = s / n, p = s - el * n;
        const int e = P.elist[w.first + el];
        const int64_t o = m.off[e];
        double* T = smem + (int64_t)el * 15 * n;
        for (int i = 0; i < 3; ++i) {
          double ja = metric<AFFINE>(m.metric, e, o, n, p, 3 * i + c);
          for (int v = 0; v < 5; ++v) T[(i * 5 + v) * n + p] = ja * P.q[5 * o + v * n + p];
        }
      }
      __syncthreads();
      for (int s = threadIdx.x; s < slots; s += blockDim.x) {
        const int el = s / n, p = s - el * n;
        const int e = P.elist[w.first + el];
        const int64_t o = m.off[e];
        const int i = p % n1, j = (p / n1) % n2, k = p / (n1 * n2);
        const double* T = smem + (int64_t)el * 15 * n;
        double acc[5];
        div_tile<5>(T, n1, n2, n3, i, j, k, D1, D2, D3, acc);
        if (!P.isolated) {
          const double* sb = P.surfq + 15 * m.soff[e];
          auto lift = [&](int f, int a, int b, int dir, double sgn, double inv_w) {
            int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3;
            int nf = na * nb;
            const double* S = sb + 15 * face_offset(n1, n2, n3, f);
            for (int v = 0; v < 5; ++v)
              acc[v] += sgn * (S[(v * 3 + c) * nf + a + na * b] - T[(dir * 5 + v) * n + p]) * inv_w;
          };
          if (i == 0) lift(0, j, k, 0, -1.0, 0.5 * w.n1 * (w.n1 + 1));
          if (i == n1 - 1) lift(1, j, k, 0, 1.0, 0.5 * w.n1 * (w.n1 + 1));
          if (j == 0) lift(2, i, k, 1, -1.0, 0.5 * w.n2 * (w.n2 + 1));
          if (j == n2 - 1) lift(3, i, k, 1, 1.0, 0.5 * w.n2 * (w.n2 + 1));
          if (k == 0) lift(4, i, j, 2, -1.0, 0.5 * w.n3 * (w.n3 + 1));
          if (k == n3 - 1) lift(5, i, j, 2, 1.0, 0.5 * w.n3 * (w.n3 + 1));
        }
        const double iJ = metric<AFFINE>(m.metric, e, o, n, p, 10);
        for (int v = 0; v < 5; ++v) P.out[15 * o + (c * 5 + v) * n + p] = acc[v] * iJ;
      }
      __syncthreads();
    }
  }
}

// ----------------------------------------------------------------- CFL step
// CFL inverse time scale per node, max-reduced over the mesh:
//   s = max(s_a, s_v),  s_a = 1/(2J) sum_i (N_i+1)^2 (|J a^i . v| + c |J a^i|),
//   s_v = 1/(4J^2) sum_i (N_i+1)^4 |J a^i|^2 max(1, gamma/Pr) mu/rho  (NS).
// Affine meshes read 1/J and |J a^i| from the element record (fields 10 and
// 11..13); AXIS meshes use |J a^i . v| = J a^i_i |v_i|.
//
// The FP64 pipe is the bound of a plain FP64 pass (a division and a square
// root per node), so the reduction runs in two kernels.  dt_filter_kernel
// evaluates s in FP32 at every node and reduces its maximum M32.  dt_kernel
// evaluates it again in FP32 and only where s32 >= M32 (1 - delta) (the
// candidates, queued per warp so that the FP64 work runs on full warps) in
// FP64, whose maximum is the result.  Error bound: with the inputs truncated
// to FP32 (relative error < 2^-23 = eps32 each), every quantity of s is a
// sum of non-negative terms except the
// pressure gm1 (E - k) and |J a^i . v|.  The guard E - k >= E/16 keeps the
// pressure's relative error below ~180 eps32 and the Mach number below 7.3,
// which bounds the error of |J a^i . v| by ~75 eps32 of the c |J a^i| term;
// so |s32/s - 1| <= eta ~ 200 eps32 = 2.4e-5 at every node that passes the
// guard.  The FP64 maximiser n* then has s32(n*) >= M32 (1 - 2 eta), and
// delta = 2^-10 ~ 20 x 2 eta keeps it among the candidates, so the maximum
// equals the plain FP64 pass.  A node that fails the guard, or whose FP32
// value is not finite, is always a candidate (and so still raises the
// non-physical flag through its FP64 value).
constexpr float kDtMargin = 1.0f / 1024.0f;

__device__ __forceinline__ float tfmax(float a, float b) { return fmaxf(a, b); }
__device__ __forceinline__ double tfmax(double a, double b) { return fmax(a, b); }

// A double as a float by integer operations on its bits (the FP64 pipe,
// which also converts, is the scarce one): the magnitude bits clamped to the
// float exponent range, rebiased and shifted, the mantissa truncated to 23
// bits (relative error below 2^-23 in the normal float range).  Magnitudes
// below it come out below 2^-126; magnitudes above it, infinities and NaNs
// come out infinite or NaN, which fails the guard or the finiteness test.
template <typename T>
__device__ __forceinline__ T from_double(double x);
template <>
__device__ __forceinline__ double from_double<double>(double x) { return x; }
template <>
__device__ __forceinline__ float from_double<float>(double x) {
  const unsigned hi = (unsigned)__double2hiint(x), lo = (unsigned)__double2loint(x);
  const unsigned a = min(max(hi & 0x7fffffffu, 896u << 20), 1151u << 20);
  return __uint_as_float((hi & 0x80000000u) | ((a - (896u << 20)) << 3) | (lo >> 29));
}

// The FP32 reciprocal and square root are the approximate hardware forms
// (a few ulp, against the ~200 eps32 budget above); for x = 0 or outside
// [2^-126, 2^126] they give 0, infinity or NaN, which the guard or the
// finiteness test turns into a candidate.
__device__ __forceinline__ float recip(float x) { return __fdividef(1.0f, x); }
__device__ __forceinline__ double recip(double x) { return 1.0 / x; }
__device__ __forceinline__ float tsqrt(float x) { return x * rsqrtf(x); }
__device__ __forceinline__ double tsqrt(double x) { return sqrt(x); }
__device__ __forceinline__ float tabs(float x) { return fabsf(x); }
__device__ __forceinline__ double tabs(double x) { return fabs(x); }

// s of node p of element e (offset o, n nodes, nn = N_i + 1) in precision T;
// ok: the FP32 guard above (1e-30 < rho < 1e30, E - k >= E/16)
// a metric field in precision T: affine meshes read FP32 from the rounded copy
template <bool AFFINE, typename T>
__device__ __forceinline__ T metric_t(const MeshView& m, const float* M32, int e, int64_t o, int n, int p, int f) {
  if constexpr (AFFINE && sizeof(T) == sizeof(float)) return __ldg(M32 + kAffStride * e + f);
  else return from_double<T>(metric<AFFINE>(m.metric, e, o, n, p, f));
}

template <bool AFFINE, bool AXIS, typename T>
__device__ __forceinline__ T node_scale(const MeshView& m, const ScaleConst<T>& K, const float* M32,
                                        const double* __restrict__ Q, int e, int64_t o, int n, int p, const int nn[3],
                                        bool* ok) {
  const T gm1 = K.gm1, gamma = K.gamma;
  T q[5];
  for (int v = 0; v < 5; ++v) q[v] = from_double<T>(Q[5 * o + v * n + p]);
  const T ir = recip(q[0]);
  const T u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  const T k = T(0.5) * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]);
  *ok = q[0] > T(1e-30) && q[0] < T(1e30) && q[4] - k >= T(0.0625) * q[4];
  const T pr = gm1 * (q[4] - k);
  const T c = tsqrt(gamma * pr * ir);
  const T iJ = metric_t<AFFINE, T>(m, M32, e, o, n, p, 10);
  T sa = T(0), sv = T(0);
  for (int i = 0; i < 3; ++i) {
    const T k2 = T(nn[i] * nn[i]);
    T un, a;
    if (AXIS) {
      a = metric_t<true, T>(m, M32, e, 0, n, p, 4 * i);
      un = a * tabs(u[i]);
    } else {
      T ja[3];
      for (int d = 0; d < 3; ++d) ja[d] = metric_t<AFFINE, T>(m, M32, e, o, n, p, 3 * i + d);
      un = tabs(ja[0] * u[0] + ja[1] * u[1] + ja[2] * u[2]);
      a = AFFINE ? metric_t<true, T>(m, M32, e, 0, n, p, 11 + i) : tsqrt(ja[0] * ja[0] + ja[1] * ja[1] + ja[2] * ja[2]);
    }
    sa += k2 * (un + c * a);
    sv += k2 * k2 * a * a;
  }
  T sm = T(0.5) * iJ * sa;
  if (K.ns) {
    const T nu = K.mu * ir * K.gpr;
    sm = tfmax(sm, T(0.25) * iJ * iJ * sv * nu);
  }
  return sm;
}

template <bool AFFINE, bool AXIS>
__global__ void __launch_bounds__(kVolThreads) dt_filter_kernel(VolParams P, unsigned* m32_bits) {
  __shared__ float red[kVolThreads / 32];
  const MeshView& m = P.m;
  float smax = 0.0f;
  for (int it = blockIdx.x; it < P.n_items; it += gridDim.x) {
    WorkItem w;
    if (!take_item(P.m, P.items, P.ilist ? P.ilist[it] : it, P.n_items_all, P.elist, 0, w)) continue;
    const int nn[3] = {w.n1 + 1, w.n2 + 1, w.n3 + 1};
    const int n = nn[0] * nn[1] * nn[2];
    for (int s = threadIdx.x; s < w.count * n; s += blockDim.x) {
      const int el = fdiv(s, n), p = s - el * n;
      const int e = P.elist[w.first + el];
      bool ok;
      const float v = node_scale<AFFINE, AXIS, float>(m, P.k32, P.metric32, P.q, e, m.off[e], n, p, nn, &ok);
      if (ok && v <= FLT_MAX) smax = fmaxf(smax, v);
    }
  }
  for (int off = 16; off > 0; off >>= 1) smax = fmaxf(smax, __shfl_xor_sync(0xffffffffu, smax, off));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = smax;
  __syncthreads();
  if (threadIdx.x == 0) {
    float b = 0.0f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) b = fmaxf(b, red[i]);
    atomicMax(m32_bits, __float_as_uint(b));   // non-negative floats order like their bit patterns
  }
}

// the FP64 s of a candidate as its bit pattern (non-negative doubles order
// like their bits, so the maxima below run on the integer pipes); a NaN is
// left out of the maximum (0) and, like an infinity, raises the flag
template <bool AFFINE, bool AXIS>
__device__ __forceinline__ unsigned long long exact_scale_bits(const VolParams& P, int2 ep) {
  const MeshView& m = P.m;
  int nn[3];
  orders_of(m, ep.x, nn[0], nn[1], nn[2]);
  bool ok;
  const double sm =
      node_scale<AFFINE, AXIS, double>(m, P.k64, nullptr, P.q, ep.x, m.off[ep.x], nn[0] * nn[1] * nn[2], ep.y, nn, &ok);
  if (!(sm <= DBL_MAX)) atomicOr(P.err, 1u);
  const unsigned long long b = (unsigned long long)__double_as_longlong(sm);
  return (b & 0x7fffffffffffffffull) > 0x7ff0000000000000ull ? 0ull : b;
}

template <bool AFFINE, bool AXIS>
__global__ void __launch_bounds__(kVolThreads) dt_kernel(VolParams P, const unsigned* m32_bits,
                                                         unsigned long long* smax_bits) {
  constexpr int kWarps = kVolThreads / 32;
  __shared__ int2 queue[kWarps][64];          // candidates (element, node) of each warp
  __shared__ unsigned long long red[kWarps];
  const MeshView& m = P.m;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const float thr = __uint_as_float(*m32_bits) * (1.0f - kDtMargin);
  int cnt = 0;                                 // queued candidates (warp-uniform, < 32 between iterations)
  unsigned long long smax = 0;                 // bits of the largest FP64 s seen
  for (int it = blockIdx.x; it < P.n_items; it += gridDim.x) {
    WorkItem w;
    if (!take_item(P.m, P.items, P.ilist ? P.ilist[it] : it, P.n_items_all, P.elist, 0, w)) continue;
    const int nn[3] = {w.n1 + 1, w.n2 + 1, w.n3 + 1};
    const int n = nn[0] * nn[1] * nn[2];
    const int total = w.count * n;
    for (int base = warp * 32; base < total; base += blockDim.x) {   // warp-uniform trip count
      const int s = base + lane;
      bool cand = false;
      int e = 0, p = 0;
      if (s < total) {
        const int el = fdiv(s, n);
        p = s - el * n;
        e = P.elist[w.first + el];
        bool ok;
        const float v = node_scale<AFFINE, AXIS, float>(m, P.k32, P.metric32, P.q, e, m.off[e], n, p, nn, &ok);
        cand = !ok || !(v < thr);
        if (AFFINE && cand && p > 0) {
          // on a straight-sided element s depends on the node's state alone:
          // a node whose state equals the first node's bit for bit has its s,
          // and the first node is a candidate too (a uniform region otherwise
          // queues every node of its elements for the FP64 pass)
          const double* qe = P.q + 5 * m.off[e];
          bool same = true;
          for (int v5 = 0; v5 < 5; ++v5)
            same = same && __double_as_longlong(qe[v5 * n + p]) == __double_as_longlong(qe[v5 * n]);
          cand = !same;
        }
      }
      const unsigned mask = __ballot_sync(0xffffffffu, cand);
      if (cand) queue[warp][cnt + __popc(mask & ((1u << lane) - 1u))] = make_int2(e, p);
      cnt += __popc(mask);
      __syncwarp();
      if (cnt >= 32) {
        smax = max(smax, exact_scale_bits<AFFINE, AXIS>(P, queue[warp][lane]));
        __syncwarp();
        if (lane < cnt - 32) queue[warp][lane] = queue[warp][32 + lane];
        cnt -= 32;
        __syncwarp();
      }
    }
  }
  if (lane < cnt) smax = max(smax, exact_scale_bits<AFFINE, AXIS>(P, queue[warp][lane]));
  for (int off = 16; off > 0; off >>= 1) smax = max(smax, __shfl_xor_sync(0xffffffffu, smax, off));
  if (lane == 0) red[warp] = smax;
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned long long b = 0;
    for (int i = 0; i < kWarps; ++i) b = max(b, red[i]);
    atomicMax(smax_bits, b);
  }
}

__global__ void dt_finalize(const unsigned long long* smax_bits, double cfl, double* dt) {
  double s = __longlong_as_double((long long)*smax_bits);
  *dt = cfl / s;
}

// ----------------------------------------------------------------- tau sweep
template <typename T>
__device__ __forceinline__ T tmax(T a, T b) { return a > b ? a : b; }

template <typename T>
struct TauParams {
  MeshView m;
  int n_elem;
  const double* q;
  const double* rp;         // R^P (state layout) or null
  const int32_t* sweep;     // [n_sweep][3] (device)
  int n_sweep;
  const T* basis;           // tables in precision T
  const T* metric;          // affine: [e][kAffStride]; curved: tau geometry bank [10][n_N] per combo
  const int64_t* bank_off;  // curved: per-element bank offset (in T elements)
  T* map_new;
  T* map_trad;
  int accumulate;
  int S;                    // shared-memory buffer stride (max n_P of the size class)
  const WorkItem* items;    // tiles of same-order elements (the volume work items)
  const int32_t* elist;     // their element list
  const int32_t* ilist;     // prologue: items of this launch (one shared-memory size class)
  const int4* units;        // sweep: (item, first group, group count) units of this launch: groups of one N3
  const int4* groups;       // sweep entries grouped by (N2, N3): N2, N3, first, count
  const int2* gentries;     // group entries: sweep index, N1
  int n_list;
  T* rp_scratch;            // isolated R^P at P, state layout, when rp is null
  T gamma, mu, Pr, Rgas, kappa_R;
  double gamma64;           // gamma in FP64 (the FP32 sweep's reference records)
  int compact;              // shared-memory layout with A3 and A1 aliased (units of one group only)
  unsigned* err;
  int n_items_all, n_groups, n_gentries;   // lengths of items, groups and gentries
};

// a tau tile inside its class's shared-memory capacity S (nodes at P)
__device__ __forceinline__ bool bad_tile(const MeshView& m, const WorkItem& w, int S) {
#ifdef DG_BOUNDS_CHECK
  const bool bad = (int64_t)w.count * (w.n1 + 1) * (w.n2 + 1) * (w.n3 + 1) > S;
  if (bad && threadIdx.x == 0) flag_index(m);
  return bad;
#else
  (void)m;
  (void)w;
  (void)S;
  return false;
#endif
}

// a sweep group of a tile: coarse orders (N2, N3) within the tile's and
// entries (sweep index, N1) inside the lists (block-uniform values)
template <typename T>
__device__ __forceinline__ bool bad_group(const TauParams<T>& P, const WorkItem& w, int gi) {
#ifdef DG_BOUNDS_CHECK
  bool bad = (unsigned)gi >= (unsigned)P.n_groups;
  if (!bad) {
    const int4 g = P.groups[gi];
    bad = g.x < 1 || g.x > w.n2 || g.y < 1 || g.y > w.n3 || g.z < 0 || g.w < 0 || g.z > P.n_gentries - g.w;
    for (int k = 0; !bad && k < g.w; ++k) {
      const int2 ent = P.gentries[g.z + k];
      bad = (unsigned)ent.x >= (unsigned)P.n_sweep || ent.y < 1 || ent.y > DG_MAX_ORDER;
    }
  }
  if (bad && threadIdx.x == 0) flag_index(P.m);
  return bad;
#else
  (void)P;
  (void)w;
  (void)gi;
  return false;
#endif
}

// offset (in nodes) of the metrics of coarse orders (N1,N2,N3) inside an
// element's bank (all combos N <= P, N1 fastest, then N2, then N3)
__device__ __forceinline__ int64_t bank_combo_offset(int P1, int P2, int N1, int N2, int N3) {
  auto Sk = [](int k) { return (int64_t)k * (k + 3) / 2; };  // sum_{a=1..k} (a+1)
  int64_t s1 = Sk(P1), s2 = Sk(P2);
  return s1 * s2 * Sk(N3 - 1) + s1 * Sk(N2 - 1) * (N3 + 1) + Sk(N1 - 1) * (int64_t)(N2 + 1) * (N3 + 1);
}

template <typename T>
__device__ __forceinline__ void euler_fluxes(T gm1, const T q[5], T f[3][5]) {
  T ir = (T)1 / q[0];
  T u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  T pr = gm1 * (q[4] - (T)0.5 * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
  for (int d = 0; d < 3; ++d) {
    f[d][0] = q[1 + d];
    f[d][1] = q[1] * u[d];
    f[d][2] = q[2] * u[d];
    f[d][3] = q[3] * u[d];
    f[d][1 + d] += pr;
    f[d][4] = u[d] * (q[4] + pr);
  }
}

// Navier-Stokes viscous flux of the tau sweep from the primitive variables
// (1/rho, u, p) and the gradient g[v*3+c] = d q_v / d x_c.
template <typename T>
__device__ void viscous_prim(const TauParams<T>& P, T ir, const T u[3], T pr, const T g[15], T fv[3][5]) {
  T gm1 = P.gamma - (T)1;
  T pir = pr * ir;
  T half_u2 = (T)0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  T du[3][3], dT[3];
  for (int c = 0; c < 3; ++c) {
    for (int i = 0; i < 3; ++i) du[i][c] = (g[(1 + i) * 3 + c] - u[i] * g[c]) * ir;
    T dpc = gm1 * (g[12 + c] - (u[0] * g[3 + c] + u[1] * g[6 + c] + u[2] * g[9 + c]) + half_u2 * g[c]);
    dT[c] = (dpc - pir * g[c]) * ir;
  }
  T div = du[0][0] + du[1][1] + du[2][2];
  for (int d = 0; d < 3; ++d) {
    T tau[3];
    for (int i = 0; i < 3; ++i) tau[i] = P.mu * (du[i][d] + du[d][i]) - (i == d ? (T)(2.0 / 3.0) * P.mu * div : (T)0);
    fv[d][0] = 0;
    fv[d][1] = tau[0];
    fv[d][2] = tau[1];
    fv[d][3] = tau[2];
    fv[d][4] = u[0] * tau[0] + u[1] * tau[1] + u[2] * tau[2] + P.kappa_R * dT[d];
  }
}

template <typename T>
__device__ void viscous_t(const TauParams<T>& P, const T q[5], const T g[15], T fv[3][5]) {
  T gm1 = P.gamma - (T)1;
  T ir = (T)1 / q[0];
  T u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  T pr = gm1 * (q[4] - (T)0.5 * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
  viscous_prim(P, ir, u, pr, g, fv);
}

template <typename T>
__device__ __forceinline__ T met_at(const T* met, bool affine, int n, int p, int mm) {
  return affine ? met[mm] : met[mm * n + p];
}

// sum-factorised GL derivative of a [3][5][n] tile at node p
template <typename T>
__device__ __forceinline__ void div5(const T* basis, const T* F, int n1, int n2, int n3, int p, T acc[5]) {
  const int n = n1 * n2 * n3;
  const int pj = fdiv(p, n1), k = fdiv(pj, n2), i = p - pj * n1, j = pj - k * n2;
  const T* D1 = basis + c_boff.D[n1 - 1];
  const T* D2 = basis + c_boff.D[n2 - 1];
  const T* D3 = basis + c_boff.D[n3 - 1];
  for (int v = 0; v < 5; ++v) acc[v] = 0;
  int b1 = n1 * (j + n2 * k), b2 = i + n1 * n2 * k, b3 = i + n1 * j;
  for (int mm = 0; mm < n1; ++mm) {
    T d = D1[i * n1 + mm];
    for (int v = 0; v < 5; ++v) acc[v] += d * F[(0 * 5 + v) * n + b1 + mm];
  }
  for (int mm = 0; mm < n2; ++mm) {
    T d = D2[j * n2 + mm];
    for (int v = 0; v < 5; ++v) acc[v] += d * F[(1 * 5 + v) * n + b2 + n1 * mm];
  }
  for (int mm = 0; mm < n3; ++mm) {
    T d = D3[k * n3 + mm];
    for (int v = 0; v < 5; ++v) acc[v] += d * F[(2 * 5 + v) * n + b3 + n1 * n2 * mm];
  }
}

// apply a (t x f) matrix along direction dir of an [nvar][e0 e1 e2] tile
template <typename T>
__device__ void apply_dir_tile(const T* A, int t, int f, int dir, int e0, int e1, int e2, const T* in, int sin_,
                               T* out, int sout, int nvar) {
  int o0 = e0, o1 = e1, o2 = e2;
  if (dir == 0) o0 = t; else if (dir == 1) o1 = t; else o2 = t;
  const int no = o0 * o1 * o2;
  for (int p = threadIdx.x; p < no; p += blockDim.x) {
    const int pj = fdiv(p, o0), k = fdiv(pj, o1), i = p - pj * o0, j = pj - k * o1;
    int r, base, stride;
    if (dir == 0) { r = i; base = e0 * (j + e1 * k); stride = 1; }
    else if (dir == 1) { r = j; base = i + e0 * e1 * k; stride = e0; }
    else { r = k; base = i + e0 * j; stride = e0 * e1; }
    for (int c = 0; c < nvar; ++c) {
      T acc = 0;
      for (int mm = 0; mm < f; ++mm) acc += A[r * f + mm] * in[c * sin_ + base + mm * stride];
      out[c * sout + p] = acc;
    }
  }
  __syncthreads();
}

template <typename T>
__device__ __forceinline__ void block_max2(T& a, T& b, T (*red)[kTauThreads / 32]) {
  for (int o = 16; o > 0; o >>= 1) {
    a = tmax(a, __shfl_xor_sync(0xffffffffu, a, o));
    b = tmax(b, __shfl_xor_sync(0xffffffffu, b, o));
  }
  if ((threadIdx.x & 31) == 0) {
    red[0][threadIdx.x >> 5] = a;
    red[1][threadIdx.x >> 5] = b;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int i = 1; i < (int)(blockDim.x >> 5); ++i) {
      a = tmax(a, red[0][i]);
      b = tmax(b, red[1][i]);
    }
  }
}

template <typename T>
__device__ __forceinline__ void map_store(T* map, int64_t idx, int accumulate, T v) {
  if (!map) return;
  map[idx] = accumulate ? tmax(map[idx], v) : v;
}

template <typename T>
__device__ __forceinline__ T mul_rn(T a, T b);
template <>
__device__ __forceinline__ float mul_rn<float>(float a, float b) { return __fmul_rn(a, b); }
template <>
__device__ __forceinline__ double mul_rn<double>(double a, double b) { return __dmul_rn(a, b); }

// non-negative floating-point values order like their bit patterns
__device__ __forceinline__ void smax_bits(unsigned int* slot, float v) { atomicMax(slot, __float_as_uint(v)); }
__device__ __forceinline__ void smax_bits(unsigned long long* slot, double v) {
  atomicMax(slot, (unsigned long long)__double_as_longlong(v));
}
// Both norms of a warp's items into their slots (all 32 lanes call it;
// slot < 0: the lane has no item).  FP32: the lanes of one slot reduce their
// maxima first and one of them makes the atomic, since the items of a warp
// mostly belong to one or two elements (32 atomics on one address serialise).
// The maxima are taken over the bit patterns of nonnegative values.
__device__ __forceinline__ void warp_norm_max(unsigned* na, unsigned* nb, int slot, float a, float b) {
  const unsigned peers = __match_any_sync(0xffffffffu, slot);
  const unsigned ma = __reduce_max_sync(peers, __float_as_uint(a));
  const unsigned mb = __reduce_max_sync(peers, __float_as_uint(b));
  if (slot >= 0 && (int)(threadIdx.x & 31) == __ffs(peers) - 1) {
    atomicMax(na + slot, ma);
    atomicMax(nb + slot, mb);
  }
}
__device__ __forceinline__ void warp_norm_max(unsigned long long* na, unsigned long long* nb, int slot, double a,
                                              double b) {
  if (slot >= 0) {
    smax_bits(na + slot, a);
    smax_bits(nb + slot, b);
  }
}
template <typename T>
struct Bits;
template <>
struct Bits<float> {
  typedef unsigned int type;
  static __device__ __forceinline__ float val(type b) { return __uint_as_float(b); }
};
template <>
struct Bits<double> {
  typedef unsigned long long type;
  static __device__ __forceinline__ double val(type b) { return __longlong_as_double((long long)b); }
};

// metrics of tile element el at coarse orders (N1,N2,N3) (P: its own orders)
template <typename T, bool AFFINE>
__device__ __forceinline__ const T* tile_met(const TauParams<T>& P, int e, int P1, int P2, int N1, int N2, int N3) {
  if (AFFINE) return P.metric + kAffStride * (int64_t)e;
  return P.metric + P.bank_off[e] + 10 * bank_combo_offset(P1, P2, N1, N2, N3);
}

// The FP32 sweep works on deviations from a per-element reference state, the
// state at the element's first node, q_r (FP64).  A flux field that is
// constant over the element has zero divergence: the rows of the GL
// derivative sum to zero and the curl-form metrics satisfy the discrete
// metric identities (sum_i D_i (J a^i) = 0).  So R^N(I q) is unchanged, in exact
// arithmetic, when the constant f(q_r) is taken out of every flux, and the
// restriction reproduces constants, so I q = q_r + I (q - q_r).  The FP32
// arithmetic then rounds relative to the deviations q' = q - q_r (formed in
// FP64) and to the flux deviations f(q) - f(q_r), not to the state itself: at
// Mach 0.1 the pressure p ~ 143 and the energy flux ~ 500 u of the pulse
// otherwise put a floor of FP32 rounding under every tau.
// Reference record (FP32 values formed in FP64): rho_r, u_f (the reference
// velocity rounded to FP32), m_r, c0 = m_r - u_f rho_r, c1 = (gamma-1) E_r -
// (gamma-1)/2 rho_r |u_f|^2 - p_f, h_f = E_r + p_f, |u_f|^2, p_f (the
// reference pressure rounded to FP32).  With rho = rho_r + rho',
//   u - u_f  = (c0 + m' - u_f rho') / rho,
//   p - p_f  = c1 + (gamma-1) (E' - rho' |u_f|^2 / 2 - rho (u_f.u' + |u'|^2/2)),
// and the flux deviations (the constants m_r,d, m_r u_f,d + p_f, h u_f,d
// dropped): mass m'_d, momentum m_r u'_d + m' u_d + p' e_d, energy
// h u'_d + (E' + p') u_d.
enum { kRefRho = 0, kRefU = 1, kRefM = 4, kRefC0 = 7, kRefC1 = 10, kRefH = 11, kRefU2 = 12, kRefP = 13 };

// The reference record of an element from its first node (state layout at
// q + 5 off_e, n nodes), in FP64.
__device__ __forceinline__ void tau_ref_make(const double* q, int n, double gm1, float* ref) {
  const double r = q[0], E = q[4 * n];
  const double m[3] = {q[n], q[2 * n], q[3 * n]};
  double uf[3], u2 = 0.0, mu = 0.0;
  for (int c = 0; c < 3; ++c) {
    const float f = (float)(m[c] / r);
    uf[c] = f;
    u2 += uf[c] * uf[c];
    mu += m[c] * m[c];
    ref[kRefU + c] = f;
    ref[kRefM + c] = (float)m[c];
    ref[kRefC0 + c] = (float)(m[c] - uf[c] * r);
  }
  const float pf = (float)(gm1 * (E - 0.5 * mu / r));
  ref[kRefRho] = (float)r;
  ref[kRefC1] = (float)(gm1 * E - 0.5 * gm1 * r * u2 - (double)pf);
  ref[kRefH] = (float)(E + (double)pf);
  ref[kRefU2] = (float)u2;
  ref[kRefP] = pf;
}

// Primitive variables of the deviation form at one node: 1/rho, u (full),
// u' = u - u_f and p' = p - p_f from the deviations d = q - q_r.
__device__ __forceinline__ void dev_primitive(float gm1, const float d[5], const float* ref, float& ir, float u[3],
                                              float ud[3], float& pd) {
  const float rho = ref[kRefRho] + d[0];
  ir = 1.0f / rho;
  float uu = 0.0f, u2 = 0.0f;
  for (int c = 0; c < 3; ++c) {
    ud[c] = (ref[kRefC0 + c] + d[1 + c] - ref[kRefU + c] * d[0]) * ir;
    u[c] = ref[kRefU + c] + ud[c];
    uu += ref[kRefU + c] * ud[c];
    u2 += ud[c] * ud[c];
  }
  pd = ref[kRefC1] + gm1 * (d[4] - 0.5f * d[0] * ref[kRefU2] - rho * (uu + 0.5f * u2));
}

// Euler flux deviations f_d(q) - f_d(q_r) at one node (deviation form above)
// from the node's primitive deviations.
__device__ __forceinline__ void dev_fluxes(const float d[5], const float* ref, const float u[3], const float ud[3],
                                           float pd, float f[3][5]) {
  const float ep = d[4] + pd;
  for (int k = 0; k < 3; ++k) {
    f[k][0] = d[1 + k];
    for (int c = 0; c < 3; ++c) f[k][1 + c] = ref[kRefM + c] * ud[k] + d[1 + c] * u[k];
    f[k][1 + k] += pd;
    f[k][4] = ref[kRefH] * ud[k] + ep * u[k];
  }
}

__device__ __forceinline__ void euler_fluxes_dev(float gm1, const float d[5], const float* ref, float f[3][5]) {
  float ir, u[3], ud[3], pd;
  dev_primitive(gm1, d, ref, ir, u, ud, pd);
  dev_fluxes(d, ref, u, ud, pd, f);
}

// Contravariant Euler fluxes Ft^i = J a^i . f at one node into F (stride n):
// the tau sweep's one flux routine, shared by R^P and every coarse residual so
// that R^N at N = P reproduces R^P bit for bit (tau at N = P is then exactly
// 0).  AXIS: J a^i = (J a^i_i) e_i.
template <typename T, bool AFFINE, bool AXIS>
__device__ __forceinline__ void tau_flux(T gm1, const T* met, int n, int p, const T q[5], const float* ref, T* F) {
  T f[3][5];
  if constexpr (std::is_same<T, float>::value) euler_fluxes_dev(gm1, q, ref, f);   // q: deviations q - q_r
  else euler_fluxes(gm1, q, f);
  for (int i = 0; i < 3; ++i) {
    if (AXIS) {
      const T a = met_at(met, AFFINE, n, p, 4 * i);
      for (int v = 0; v < 5; ++v) F[(i * 5 + v) * n] = a * f[i][v];
    } else {
      const T ja0 = met_at(met, AFFINE, n, p, 3 * i), ja1 = met_at(met, AFFINE, n, p, 3 * i + 1),
              ja2 = met_at(met, AFFINE, n, p, 3 * i + 2);
      for (int v = 0; v < 5; ++v) F[(i * 5 + v) * n] = ja0 * f[0][v] + ja1 * f[1][v] + ja2 * f[2][v];
    }
  }
}

// The per-node pieces of the isolated residual, shared by R^P and every
// coarse residual of the sweep so that R^N at N = P reproduces R^P bit for
// bit.  Element tiles are [field][n]; met is the element's metric block.
// BR1 gradient, component c: the contravariant fluxes J a^i_c q of the state.
template <typename T, bool AFFINE>
__device__ __forceinline__ void tau_grad_flux(const T* met, int n, int p, int c, const T* X, T* F) {
  for (int i = 0; i < 3; ++i) {
    const T ja = met_at(met, AFFINE, n, p, 3 * i + c);
    for (int v = 0; v < 5; ++v) F[(i * 5 + v) * n + p] = ja * X[v * n + p];
  }
}

// ... their GL divergence over J: component c of the gradient, G[v*3+c]
template <typename T, bool AFFINE>
__device__ __forceinline__ void tau_grad_store(const T* basis, const T* met, int n1, int n2, int n3, int p, int c,
                                               const T* F, T* G) {
  const int n = n1 * n2 * n3;
  T acc[5];
  div5(basis, F, n1, n2, n3, p, acc);
  const T iJ = (T)1 / met_at(met, AFFINE, n, p, 9);
  for (int v = 0; v < 5; ++v) G[(v * 3 + c) * n + p] = acc[v] * iJ;
}

// Navier-Stokes contravariant fluxes J a^i . (f - f_v) at node p
template <typename T, bool AFFINE>
__device__ __forceinline__ void tau_ns_flux(const TauParams<T>& P, T gm1, const T* met, int n, int p, const T q[5],
                                            const float* ref, const T* G, T* F) {
  T f[3][5];
  T g[15], fv[3][5];
  for (int c = 0; c < 15; ++c) g[c] = G[c * n + p];
  if constexpr (std::is_same<T, float>::value) {   // q: deviations q - q_r; G: the gradient of q - q_r, that of q
    float ir, u[3], ud[3], pd;
    dev_primitive(gm1, q, ref, ir, u, ud, pd);
    dev_fluxes(q, ref, u, ud, pd, f);
    viscous_prim(P, ir, u, ref[kRefP] + pd, g, fv);
  } else {
    euler_fluxes(gm1, q, f);
    viscous_t(P, q, g, fv);
  }
  for (int d = 0; d < 3; ++d)
    for (int v = 0; v < 5; ++v) f[d][v] -= fv[d][v];
  for (int i = 0; i < 3; ++i) {
    const T ja0 = met_at(met, AFFINE, n, p, 3 * i), ja1 = met_at(met, AFFINE, n, p, 3 * i + 1),
            ja2 = met_at(met, AFFINE, n, p, 3 * i + 2);
    for (int v = 0; v < 5; ++v) F[(i * 5 + v) * n + p] = ja0 * f[0][v] + ja1 * f[1][v] + ja2 * f[2][v];
  }
}

// R = -(1/J) div F at node p, rounded as when stored
template <typename T, bool AFFINE>
__device__ __forceinline__ void tau_node_residual(const T* basis, const T* met, int n1, int n2, int n3, int p,
                                                  const T* F, T r[5], T& J) {
  const int n = n1 * n2 * n3;
  T acc[5];
  div5(basis, F, n1, n2, n3, p, acc);
  J = met_at(met, AFFINE, n, p, 9);
  const T iJ = -(T)1 / J;
  for (int v = 0; v < 5; ++v) r[v] = mul_rn(acc[v], iJ);
}

// Both tau norms at node p of the coarse grid (c1, c2, c3): tau~ = I R^P - R^N
// (IR: I R^P, [5][n]), max |tau~| and max |J w tau~| into a, b
template <typename T, bool AFFINE>
__device__ __forceinline__ void tau_node_norms(const T* basis, const T* met, int c1, int c2, int c3, int p,
                                               const T* F, const T* IR, const T* w1, const T* w2, const T* w3,
                                               T& a, T& b) {
  const int n = c1 * c2 * c3;
  T r[5], J;
  tau_node_residual<T, AFFINE>(basis, met, c1, c2, c3, p, F, r, J);
  const int pj = fdiv(p, c1), k = fdiv(pj, c2), i = p - pj * c1, j = pj - k * c2;
  const T Jw = J * w1[i] * w2[j] * w3[k];
  a = 0;
  b = 0;
  for (int v = 0; v < 5; ++v) {
    const T d = IR[v * n + p] - r[v];   // tau~ = I R^P - R^N(I q^P)
    a = tmax(a, (T)fabs(d));
    b = tmax(b, (T)fabs(Jw * d));
  }
}

// Isolated residual R^P of a tile of cnt same-order elements, state X[el][5][n]
// (element stride xs) at orders (n1,n2,n3): R = -(1/J) sum_i D^(i) Ft^i, with
// the element-local BR1 gradient and viscous flux for Navier-Stokes; element
// e's R to Rout + 5*off_e, [5][n].
template <typename T, bool AFFINE, bool NS, bool AXIS>
__device__ void tau_tile_residual(const TauParams<T>& P, const int32_t* els, int cnt, int P1, int P2, int N1, int N2,
                                  int N3, const T* X, int xs, const float* refs, T* Ft, T* Gs, T* Rout) {
  const int n1 = N1 + 1, n2 = N2 + 1, n3 = N3 + 1, n = n1 * n2 * n3, pts = cnt * n;
  const T gm1 = P.gamma - (T)1;
  const MeshView& m = P.m;
  if (NS) {
    for (int c = 0; c < 3; ++c) {
      for (int t = threadIdx.x; t < pts; t += blockDim.x) {
        const int el = fdiv(t, n), p = t - el * n;
        const T* met = tile_met<T, AFFINE>(P, els[el], P1, P2, N1, N2, N3);
        tau_grad_flux<T, AFFINE>(met, n, p, c, X + el * xs, Ft + el * 15 * n);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < pts; t += blockDim.x) {
        const int el = fdiv(t, n), p = t - el * n;
        const T* met = tile_met<T, AFFINE>(P, els[el], P1, P2, N1, N2, N3);
        tau_grad_store<T, AFFINE>(P.basis, met, n1, n2, n3, p, c, Ft + el * 15 * n, Gs + el * 15 * n);
      }
      __syncthreads();
    }
  }
  for (int t = threadIdx.x; t < pts; t += blockDim.x) {
    const int el = fdiv(t, n), p = t - el * n;
    const T* met = tile_met<T, AFFINE>(P, els[el], P1, P2, N1, N2, N3);
    T q[5];
    for (int v = 0; v < 5; ++v) q[v] = X[el * xs + v * n + p];
    const float* ref = std::is_same<T, float>::value ? refs + kTauRefStride * el : nullptr;
    if (NS) tau_ns_flux<T, AFFINE>(P, gm1, met, n, p, q, ref, Gs + el * 15 * n, Ft + el * 15 * n);
    else tau_flux<T, AFFINE, AXIS>(gm1, met, n, p, q, ref, Ft + el * 15 * n + p);
  }
  __syncthreads();
  for (int t = threadIdx.x; t < pts; t += blockDim.x) {
    const int el = fdiv(t, n), p = t - el * n;
    const int e = els[el];
    const T* met = tile_met<T, AFFINE>(P, e, P1, P2, N1, N2, N3);
    T r[5], J;
    tau_node_residual<T, AFFINE>(P.basis, met, n1, n2, n3, p, Ft + el * 15 * n, r, J);
    const int64_t o = m.off[e];
    for (int v = 0; v < 5; ++v) Rout[5 * o + v * n + p] = r[v];
  }
  __syncthreads();
}

// Element el's reference record (FP32 sweep; the FP64 sweep has none).
template <typename T>
__device__ __forceinline__ const float* tau_ref_of(const float* refs, int el) {
  return std::is_same<T, float>::value ? refs + kTauRefStride * el : nullptr;
}

// Stages a tile's q^P (fields 0..4) and, with_rp, R^P (fields 5..9) in
// shared memory, [el][10][nP] at X, read once from global memory.  FP64: the
// values as they are.  FP32: q^P as deviations from the element's
// first-node state, subtracted in FP64 before the rounding, with each
// element's reference record in refs (the deviation form of tau_ref_make);
// R^P (the isolated residual, which the constant drops out of) as it is.
template <typename T>
__device__ void tau_stage(const TauParams<T>& P, const int32_t* els, int cnt, int nP, bool with_rp, T* X,
                          float* refs) {
  constexpr bool DEV = std::is_same<T, float>::value;
  const MeshView& m = P.m;
  if (DEV)
    for (int el = threadIdx.x; el < cnt; el += blockDim.x)
      tau_ref_make(P.q + 5 * m.off[els[el]], nP, P.gamma64 - 1.0, refs + kTauRefStride * el);
  for (int t = threadIdx.x; t < cnt * nP; t += blockDim.x) {
    const int el = fdiv(t, nP), p = t - el * nP;
    const int64_t o5 = 5 * m.off[els[el]];
    const double* qe = P.q + o5;
    T* x = X + el * 10 * nP + p;
    for (int v = 0; v < 5; ++v) x[v * nP] = DEV ? (T)(qe[v * nP + p] - qe[v * nP]) : (T)qe[v * nP + p];
    if (with_rp) {
      if (P.rp)
        for (int v = 0; v < 5; ++v) x[(5 + v) * nP] = (T)P.rp[o5 + v * nP + p];
      else
        for (int v = 0; v < 5; ++v) x[(5 + v) * nP] = P.rp_scratch[o5 + v * nP + p];
    }
  }
  __syncthreads();
}

// The chunk of sweep entries [first, first + k) of a group that starts at
// entry first: entries while their items (cnt nN each, none when N1 > P1)
// fit the tile capacity S and their norm slots (cnt each) fit kVolThreads;
// one entry at least (cnt nN <= cnt nP <= S).  Returns k; total = the items.
__device__ __forceinline__ int tau_chunk(const int2* gent, int first, int n_ent, int P1, int cnt, int c23, int S,
                                         int& total) {
  int k = 0;
  total = 0;
  while (first + k < n_ent && k < kTauChunk) {
    const int M1 = gent[first + k].y;
    const int sz = M1 > P1 ? 0 : cnt * (M1 + 1) * c23;
    if (k > 0 && (total + sz > S || (k + 1) * cnt > kVolThreads)) break;
    total += sz;
    ++k;
  }
  return k;
}

// Item t of a chunk: its entry j, the entry's first item base and its N1.
__device__ __forceinline__ void tau_chunk_item(const int2* gent, int first, int t, int P1, int cnt, int c23, int& base,
                                               int& j, int& M1) {
  base = 0;
  j = 0;
  M1 = gent[first].y;
  int sz = M1 > P1 ? 0 : cnt * (M1 + 1) * c23;
  while (t >= base + sz) {
    base += sz;
    M1 = gent[first + ++j].y;
    sz = M1 > P1 ? 0 : cnt * (M1 + 1) * c23;
  }
}

// Thread 0 of the Euler sweep: the next piece of a batch's entry table, from
// group btab[2], entry btab[3] of the batch's nb groups (from group gb of
// the list): every entry with N1 <= P1, as (sweep index, N1, N2 + 1, the
// group's A2 offset), at most kTauBatchEntries; btab[1] the count, btab[2..3]
// where the next piece starts.
template <typename T>
__device__ void tau_fill_entries(const TauParams<T>& P, int gb, int nb, int P1, const int4* gtab, int4* etab,
                                 int* btab) {
  int k = 0, g = btab[2], e = btab[3];
  while (g < nb && k < kTauBatchEntries) {
    const int4 gr = P.groups[gb + g];   // N2, N3, first entry, entry count
    if (e >= gr.w) {
      ++g;
      e = 0;
      continue;
    }
    const int2 ent = P.gentries[gr.z + e];
    if (ent.y <= P1) etab[k++] = make_int4(ent.x, ent.y, gtab[g].x, gtab[g].y);
    ++e;
  }
  btab[1] = k;
  btab[2] = g;
  btab[3] = e;
}

// The chunk of table entries [first, first + k): entries while their items
// (cnt (N1+1)(N2+1) c3 each) fit the tile capacity S and their norm slots
// (cnt each) fit kVolThreads; one entry at least (its items <= cnt n_P <= S).
// Returns k; total = the items.
__device__ __forceinline__ int tau_batch_chunk(const int4* etab, int first, int n_tab, int cnt, int c3, int S,
                                               int& total) {
  int k = 0;
  total = 0;
  while (first + k < n_tab && k < kTauChunk) {
    const int4 en = etab[first + k];
    const int sz = cnt * (en.y + 1) * en.z * c3;
    if (k > 0 && (total + sz > S || (k + 1) * cnt > kVolThreads)) break;
    total += sz;
    ++k;
  }
  return k;
}

// Item t of a chunk: its entry (returned), the entry's index j in the chunk
// and the entry's first item base.
__device__ __forceinline__ int4 tau_batch_item(const int4* etab, int first, int t, int cnt, int c3, int& base,
                                               int& j) {
  base = 0;
  j = 0;
  int4 en = etab[first];
  int sz = cnt * (en.y + 1) * en.z * c3;
  while (t >= base + sz) {
    base += sz;
    en = etab[first + ++j];
    sz = cnt * (en.y + 1) * en.z * c3;
  }
  return en;
}

// Prologue of the isolated Navier-Stokes sweep (field-major tiles; the Euler
// sweep runs tau_euler_prologue_kernel), one tile per CTA iteration: the
// isolated R^P of every element (into the scratch, unless the caller gave
// R^P), and -1 in the maps for every sweep entry the element's orders cannot
// reach.
template <typename T, bool AFFINE, bool NS, bool AXIS>
__global__ void __launch_bounds__(kVolThreads) tau_prologue_kernel(TauParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float Ref[std::is_same<T, float>::value ? kTauRefElems : 1][kTauRefStride];
  T* sm = reinterpret_cast<T*>(smem_raw);
  const int S = P.S;
  T* A1 = P.compact ? sm : sm + 20 * S;
  T* Ft = sm + (P.compact ? 20 : 30) * S;
  T* Gs = Ft + 15 * S;
  for (int li = blockIdx.x; li < P.n_list; li += gridDim.x) {
    WorkItem w;
    if (!take_item(P.m, P.items, P.ilist[li], P.n_items_all, P.elist, 0, w)) continue;
    if (bad_tile(P.m, w, P.S)) continue;
    const int32_t* els = P.elist + w.first;
    const int cnt = w.count;
    const int P1 = w.n1, P2 = w.n2, P3 = w.n3, nP = (P1 + 1) * (P2 + 1) * (P3 + 1);
    for (int t = threadIdx.x; t < cnt * P.n_sweep; t += blockDim.x) {
      const int el = fdiv(t, P.n_sweep), s = t - el * P.n_sweep;
      if (P.sweep[3 * s] > P1 || P.sweep[3 * s + 1] > P2 || P.sweep[3 * s + 2] > P3) {
        const int64_t idx = (int64_t)els[el] * P.n_sweep + s;
        if (P.map_new) P.map_new[idx] = (T)-1;
        if (P.map_trad) P.map_trad[idx] = (T)-1;
      }
    }
    if (P.rp) continue;
#ifdef DG_BOUNDS_CHECK
    if (std::is_same<T, float>::value && cnt > kTauRefElems) {   // one reference record per element
      if (threadIdx.x == 0) flag_index(P.m);
      continue;
    }
#endif
    tau_stage(P, els, cnt, nP, false, A1, &Ref[0][0]);
    tau_tile_residual<T, AFFINE, NS, AXIS>(P, els, cnt, P1, P2, P1, P2, P3, A1, 10 * nP, &Ref[0][0], Ft, Gs,
                                           P.rp_scratch);
  }
}

// The isolated Navier-Stokes sweep (the Euler sweep runs tau_euler_kernel),
// one unit per CTA iteration: a tile and the groups of one N3 (a group is the
// sweep entries sharing (N2, N3)).  The unit restricts
// q^P and R^P in xi3 once, each group in xi2, then runs the group's entries
// in chunks: restriction in xi1, coarse isolated residual fused with both
// tau norms, map store.
template <typename T, bool AFFINE, bool NS, bool AXIS>
__global__ void __launch_bounds__(kVolThreads) tau_kernel(TauParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  typedef typename Bits<T>::type B;
  __shared__ B na2[2][kVolThreads], nb2[2][kVolThreads];   // per-element norms, two entries in flight
  __shared__ float Ref[std::is_same<T, float>::value ? kTauRefElems : 1][kTauRefStride];
  const int S = P.S;     // tile capacity in nodes (max count * n_P of the class)
  // [el][10][nP] q^P and R^P staged (ST); restricted in xi3 (A3: [el][10][pts3]),
  // in xi2 and xi3 (A2: [el][10][pts2]), at N (A1: [el][XF][nN], I q^P and / or
  // I R^P); fluxes Ft and (NS) gradients Gs [el][15][nN].  Layout (units of S
  // values): A3 0-10, A2 10-20, ST and A1 20-30, Ft 30-45, Gs 45-60.  The
  // compact layout (units of one group) reuses what is dead by then: A3 0-10,
  // ST 10-20 then A2, A1 0-10 once A3 is read, Ft 20-35, Gs 35-50.
  T* A3 = sm;
  T* ST = sm + (P.compact ? 10 : 20) * S;
  T* A2 = sm + 10 * S;
  T* A1 = P.compact ? sm : sm + 20 * S;
  T* Ft = sm + (P.compact ? 20 : 30) * S;
  T* Gs = Ft + 15 * S;
  const MeshView& m = P.m;
  for (int ui = blockIdx.x; ui < P.n_list; ui += gridDim.x) {
    const int4 u = P.units[ui];
    WorkItem w;
    if (!take_item(P.m, P.items, u.x, P.n_items_all, P.elist, 0, w)) continue;
    if (bad_tile(P.m, w, P.S) || bad_group(P, w, u.y)) continue;
#ifdef DG_BOUNDS_CHECK
    // one norm slot per element and chunk entry; one reference record per
    // element (FP32); the compact layout holds one group
    if (w.count > kVolThreads || (std::is_same<T, float>::value && w.count > kTauRefElems) ||
        (P.compact && u.z != 1)) {
      if (threadIdx.x == 0) flag_index(P.m);
      continue;
    }
#endif
    const int32_t* els = P.elist + w.first;
    const int cnt = w.count;
    const int P1 = w.n1, P2 = w.n2, P3 = w.n3, n1 = P1 + 1, n2 = P2 + 1, n3 = P3 + 1, nP = n1 * n2 * n3;
    const int N3 = P.groups[u.y].y, c3 = N3 + 1, n12 = n1 * n2;
    tau_stage(P, els, cnt, nP, true, ST, &Ref[0][0]);   // q^P (FP32: deviations) and R^P, once per unit
    {  // xi3, once for the unit's groups
      const T* I3 = P.basis + c_boff.I[P3][N3];
      const int per = n12 * c3;
      for (int t = threadIdx.x; t < cnt * per; t += blockDim.x) {
        const int el = fdiv(t, per), x = t - el * per, k = fdiv(x, n12), ij = x - k * n12;
        const T* src = ST + el * 10 * nP + ij;
        T acc[10];
        for (int c = 0; c < 10; ++c) acc[c] = 0;
        for (int mm = 0; mm < n3; ++mm) {
          const T wk = I3[k * n3 + mm];
          for (int c = 0; c < 10; ++c) acc[c] += wk * src[c * nP + n12 * mm];
        }
        for (int c = 0; c < 10; ++c) A3[el * 10 * per + c * per + x] = acc[c];
      }
      __syncthreads();
    }
    for (int gi = u.y; gi < u.y + u.z; ++gi) {   // the groups (N2, N3) of this N3, N2 ascending
    if (gi > u.y && bad_group(P, w, gi)) continue;
    const int4 g = P.groups[gi];      // N2, N3, first entry, entry count
    const int N2 = g.x, c2 = N2 + 1;
#ifdef DG_BOUNDS_CHECK
    if (g.y != N3) {
      if (threadIdx.x == 0) flag_index(m);
      continue;
    }
#endif
    {  // xi2
      const T* I2 = P.basis + c_boff.I[P2][N2];
      const int pin = n12 * c3, per = n1 * c2 * c3;
      for (int t = threadIdx.x; t < cnt * per; t += blockDim.x) {
        const int el = fdiv(t, per), x = t - el * per, xj = fdiv(x, n1), k = fdiv(xj, c2), i = x - xj * n1, j = xj - k * c2;
        const T* src = A3 + el * 10 * pin + i + n12 * k;
        T acc[10];
        for (int c = 0; c < 10; ++c) acc[c] = 0;
        for (int mm = 0; mm < n2; ++mm) {
          const T wj = I2[j * n2 + mm];
          for (int c = 0; c < 10; ++c) acc[c] += wj * src[c * pin + n1 * mm];
        }
        for (int c = 0; c < 10; ++c) A2[el * 10 * per + c * per + x] = acc[c];
      }
      __syncthreads();
    }
    // The group's entries in chunks of at most S coarse nodes (tau_chunk),
    // one pass per step for the whole chunk: (1) store the previous chunk's
    // norms, clear this chunk's slots, restrict in xi1 (Euler: and take the
    // fluxes); Navier-Stokes: (2-7) the BR1 gradient, (8) the fluxes; (last)
    // derivative, tau and both norms.  Entry j of a chunk owns cnt nN_j items
    // from its base and the norm slots j cnt + el; its elements' restricted
    // fields are [el][XF][nN] from XF base in A1 (Euler: I R^P; Navier-Stokes:
    // I q^P, then I R^P).
    constexpr int XF = NS ? 10 : 5;
    const T gm1 = P.gamma - (T)1;
    const T* w2 = P.basis + c_boff.W[N2];
    const T* w3 = P.basis + c_boff.W[N3];
    const int pin = n1 * c2 * c3, c23 = c2 * c3;
    const int2* gent = P.gentries + g.z;      // (sweep index, N1) per entry
    int prev_first = 0, prev_k = 0, buf = 0;
    for (int first = 0; first < g.w;) {
      int total;
      const int k = tau_chunk(gent, first, g.w, P1, cnt, c23, S, total);   // the same in every thread
      const int nsl = (prev_k > k ? prev_k : k) * cnt;
      for (int sl = threadIdx.x; sl < nsl; sl += blockDim.x) {
        const int j = fdiv(sl, cnt), el = sl - j * cnt;
        if (j < prev_k) {
          const int2 pe = gent[prev_first + j];
          if (pe.y <= P1) {
            const int64_t idx = (int64_t)els[el] * P.n_sweep + pe.x;
            map_store(P.map_new, idx, P.accumulate, Bits<T>::val(na2[buf ^ 1][sl]));
            map_store(P.map_trad, idx, P.accumulate, Bits<T>::val(nb2[buf ^ 1][sl]));
          }
        }
        if (j < k) {
          na2[buf][sl] = 0;
          nb2[buf][sl] = 0;
        }
      }
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int base, j, M1;
        tau_chunk_item(gent, first, t, P1, cnt, c23, base, j, M1);
        const int c1 = M1 + 1, nN = c1 * c23, tt = t - base;
        const int el = fdiv(tt, nN), x = tt - el * nN, jk = fdiv(x, c1), i = x - jk * c1;
        const T* I1 = P.basis + c_boff.I[P1][M1];
        const T* src = A2 + el * 10 * pin + n1 * jk;
        T acc[10];
        for (int c = 0; c < 10; ++c) acc[c] = 0;
        for (int mm = 0; mm < n1; ++mm) {
          const T wi = I1[i * n1 + mm];
          for (int c = 0; c < 10; ++c) acc[c] += wi * src[c * pin + mm];
        }
        T* X = A1 + XF * (base + el * nN) + x;
        if (NS) {
          for (int c = 0; c < 10; ++c) X[c * nN] = acc[c];
        } else {
          const T* met = tile_met<T, AFFINE>(P, els[el], P1, P2, M1, N2, N3);
          tau_flux<T, AFFINE, AXIS>(gm1, met, nN, x, acc, tau_ref_of<T>(&Ref[0][0], el),
                                    Ft + 15 * (base + el * nN) + x);
          for (int v = 0; v < 5; ++v) X[v * nN] = acc[5 + v];   // I R^P
        }
      }
      __syncthreads();
      if (NS) {
        for (int c = 0; c < 3; ++c) {
          for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int base, j, M1;
            tau_chunk_item(gent, first, t, P1, cnt, c23, base, j, M1);
            const int nN = (M1 + 1) * c23, tt = t - base, el = fdiv(tt, nN), p = tt - el * nN;
            const T* met = tile_met<T, AFFINE>(P, els[el], P1, P2, M1, N2, N3);
            tau_grad_flux<T, AFFINE>(met, nN, p, c, A1 + XF * (base + el * nN), Ft + 15 * (base + el * nN));
          }
          __syncthreads();
          for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int base, j, M1;
            tau_chunk_item(gent, first, t, P1, cnt, c23, base, j, M1);
            const int nN = (M1 + 1) * c23, tt = t - base, el = fdiv(tt, nN), p = tt - el * nN;
            const T* met = tile_met<T, AFFINE>(P, els[el], P1, P2, M1, N2, N3);
            tau_grad_store<T, AFFINE>(P.basis, met, M1 + 1, c2, c3, p, c, Ft + 15 * (base + el * nN),
                                      Gs + 15 * (base + el * nN));
          }
          __syncthreads();
        }
        for (int t = threadIdx.x; t < total; t += blockDim.x) {
          int base, j, M1;
          tau_chunk_item(gent, first, t, P1, cnt, c23, base, j, M1);
          const int nN = (M1 + 1) * c23, tt = t - base, el = fdiv(tt, nN), p = tt - el * nN;
          const T* met = tile_met<T, AFFINE>(P, els[el], P1, P2, M1, N2, N3);
          const T* X = A1 + XF * (base + el * nN);
          T q[5];
          for (int v = 0; v < 5; ++v) q[v] = X[v * nN + p];
          tau_ns_flux<T, AFFINE>(P, gm1, met, nN, p, q, tau_ref_of<T>(&Ref[0][0], el), Gs + 15 * (base + el * nN),
                                 Ft + 15 * (base + el * nN));
        }
        __syncthreads();
      }
      for (int t = threadIdx.x; t < total; t += blockDim.x) {
        int base, j, M1;
        tau_chunk_item(gent, first, t, P1, cnt, c23, base, j, M1);
        const int c1 = M1 + 1, nN = c1 * c23, tt = t - base, el = fdiv(tt, nN), p = tt - el * nN;
        const T* met = tile_met<T, AFFINE>(P, els[el], P1, P2, M1, N2, N3);
        T a, b;
        tau_node_norms<T, AFFINE>(P.basis, met, c1, c2, c3, p, Ft + 15 * (base + el * nN),
                                  A1 + XF * (base + el * nN) + (XF - 5) * nN, P.basis + c_boff.W[M1], w2, w3, a, b);
        smax_bits(na2[buf] + j * cnt + el, a);
        smax_bits(nb2[buf] + j * cnt + el, b);
      }
      __syncthreads();
      prev_first = first;
      prev_k = k;
      buf ^= 1;
      first += k;
    }
    for (int sl = threadIdx.x; sl < prev_k * cnt; sl += blockDim.x) {
      const int j = fdiv(sl, cnt), el = sl - j * cnt;
      const int2 pe = gent[prev_first + j];
      if (pe.y > P1) continue;
      const int64_t idx = (int64_t)els[el] * P.n_sweep + pe.x;
      map_store(P.map_new, idx, P.accumulate, Bits<T>::val(na2[buf ^ 1][sl]));
      map_store(P.map_trad, idx, P.accumulate, Bits<T>::val(nb2[buf ^ 1][sl]));
    }
    __syncthreads();
    }   // groups of the unit
  }
}

// ------------------------------------------------- isolated sweep, Euler
// The Euler sweep keeps its shared-memory tiles node-major: the staged and
// restricted tiles hold the 10 fields of a node (q^P or its deviations, then
// R^P) at a stride of TS values, the fluxes the 15 values J a^i . f_v of a
// node at FS, the restricted R^P at N its 5 at RS.  Every field of a node
// then sits at a fixed offset from one address.  R^P (prologue) and every R^N
// of the sweep go through the same flux and derivative routines, so that R^N
// at N = P reproduces R^P bit for bit and tau there is exactly 0.
template <typename T>
struct TauTiles {
  static constexpr int TS = 11;   // odd strides: one field of 32 consecutive nodes spans 32 banks
  static constexpr int FS = 15;
  static constexpr int RS = 5;
  // slot of J a^d . f_v within a node's flux record
  __host__ __device__ static constexpr int fo(int d, int v) { return 5 * d + v; }
};
// FP32: records of an even number of floats, each direction's five fluxes
// starting at an even slot, so that the restriction and the derivative load
// pairs of fields (8-byte shared loads; strides of 10 and 18 floats keep the
// 16 lanes of each half-warp phase on distinct banks) and run packed FP32x2
// FMAs, two fields an instruction.
template <>
struct TauTiles<float> {
  static constexpr int TS = 10;
  static constexpr int FS = 18;
  static constexpr int RS = 5;
  __host__ __device__ static constexpr int fo(int d, int v) { return 6 * d + v; }
};

// Packed FP32x2 arithmetic (sm_100 and later): two lanes of a 64-bit
// register pair, each rounded as the scalar FMA would be, so that a packed
// and a scalar sum of the same terms in the same order have the same bits.
__device__ __forceinline__ unsigned long long f2_splat(float a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %1};" : "=l"(r) : "f"(a));
  return r;
}
__device__ __forceinline__ unsigned long long f2_fma(unsigned long long a, unsigned long long b,
                                                     unsigned long long c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ unsigned long long f2_load(const float* p) {   // 8-byte aligned shared address
  return *reinterpret_cast<const unsigned long long*>(p);
}
__device__ __forceinline__ void f2_unpack(unsigned long long v, float& lo, float& hi) {
  asm("mov.b64 {%0, %1}, %2;" : "=f"(lo), "=f"(hi) : "l"(v));
}

// One output node of a restriction pass: acc[c] = sum_m w[m] src[m stride + c]
// over the nt taps m of an interpolation row w (10 fields c, node-major).
// The tap loop runs to a runtime count: one loop body for every order keeps
// the kernel's code small (fully unrolled per tap count it ran 11-19% slower,
// with more instruction-fetch stalls).
template <typename T>
__device__ __forceinline__ void restrict_node(int nt, const T* __restrict__ w, const T* src, int stride, T acc[10]) {
#pragma unroll
  for (int c = 0; c < 10; ++c) acc[c] = 0;
  for (int m = 0; m < nt; ++m) {
    const T wm = w[m];
#pragma unroll
    for (int c = 0; c < 10; ++c) acc[c] += wm * src[c];
    src += stride;
  }
}
// FP32: the ten fields as five packed pairs (src and stride even)
template <>
__device__ __forceinline__ void restrict_node<float>(int nt, const float* __restrict__ w, const float* src,
                                                     int stride, float acc[10]) {
  unsigned long long a[5];
#pragma unroll
  for (int c = 0; c < 5; ++c) a[c] = 0ull;
  for (int m = 0; m < nt; ++m) {
    const unsigned long long wm = f2_splat(w[m]);
#pragma unroll
    for (int c = 0; c < 5; ++c) a[c] = f2_fma(wm, f2_load(src + 2 * c), a[c]);
    src += stride;
  }
#pragma unroll
  for (int c = 0; c < 5; ++c) f2_unpack(a[c], acc[2 * c], acc[2 * c + 1]);
}

// acc[v] += sum_m d[m] J a^dir . f_v of the node at src + m stride, over the
// nt taps m (5 variables v; src points at node records)
template <typename T>
__device__ __forceinline__ void deriv_line(int nt, const T* __restrict__ d, const T* src, int dir, int stride,
                                           T acc[5]) {
  typedef TauTiles<T> L;
  for (int m = 0; m < nt; ++m) {
    const T dm = d[m];
#pragma unroll
    for (int v = 0; v < 5; ++v) acc[v] += dm * src[L::fo(dir, v)];
    src += stride;
  }
}
// FP32: variables (0,1) and (2,3) as packed pairs, 4 alone
template <>
__device__ __forceinline__ void deriv_line<float>(int nt, const float* __restrict__ d, const float* src, int dir,
                                                  int stride, float acc[5]) {
  typedef TauTiles<float> L;
  unsigned long long a01, a23;
  asm("mov.b64 %0, {%1, %2};" : "=l"(a01) : "f"(acc[0]), "f"(acc[1]));
  asm("mov.b64 %0, {%1, %2};" : "=l"(a23) : "f"(acc[2]), "f"(acc[3]));
  float a4 = acc[4];
  src += L::fo(dir, 0);
  for (int m = 0; m < nt; ++m) {
    const float dm = d[m];
    const unsigned long long dd = f2_splat(dm);
    a01 = f2_fma(dd, f2_load(src), a01);
    a23 = f2_fma(dd, f2_load(src + 2), a23);
    a4 = fmaf(dm, src[4], a4);
    src += stride;
  }
  f2_unpack(a01, acc[0], acc[1]);
  f2_unpack(a23, acc[2], acc[3]);
  acc[4] = a4;
}

// sum_i D^(i) Ft^i at node (i, j, k) of a c1 x c2 x c3 element whose flux
// records start at Fb (node-major, FS values a node)
template <typename T>
__device__ __forceinline__ void tau_div_nm(const T* basis, const T* Fb, int c1, int c2, int c3, int i, int j, int k,
                                           T acc[5]) {
  constexpr int FS = TauTiles<T>::FS;
#pragma unroll
  for (int v = 0; v < 5; ++v) acc[v] = 0;
  deriv_line(c1, basis + c_boff.D[c1 - 1] + i * c1, Fb + FS * (c1 * (j + c2 * k)), 0, FS, acc);
  deriv_line(c2, basis + c_boff.D[c2 - 1] + j * c2, Fb + FS * (i + c1 * c2 * k), 1, FS * c1, acc);
  deriv_line(c3, basis + c_boff.D[c3 - 1] + k * c3, Fb + FS * (i + c1 * j), 2, FS * c1 * c2, acc);
}

// The contravariant Euler fluxes J a^i . f_v at one node into its flux
// record F (FP32: the flux deviations of the deviations q in tau_flux's sense).
template <typename T, bool AFFINE, bool AXIS>
__device__ __forceinline__ void tau_flux_nm(T gm1, const T* met, int n, int p, const T q[5], const float* ref, T* F) {
  T f[3][5];
  if constexpr (std::is_same<T, float>::value) euler_fluxes_dev(gm1, q, ref, f);
  else euler_fluxes(gm1, q, f);
#pragma unroll
  for (int i = 0; i < 3; ++i) {
    if (AXIS) {
      const T a = met_at(met, AFFINE, n, p, 4 * i);
#pragma unroll
      for (int v = 0; v < 5; ++v) F[TauTiles<T>::fo(i, v)] = a * f[i][v];
    } else {
      const T ja0 = met_at(met, AFFINE, n, p, 3 * i), ja1 = met_at(met, AFFINE, n, p, 3 * i + 1),
              ja2 = met_at(met, AFFINE, n, p, 3 * i + 2);
#pragma unroll
      for (int v = 0; v < 5; ++v) F[TauTiles<T>::fo(i, v)] = ja0 * f[0][v] + ja1 * f[1][v] + ja2 * f[2][v];
    }
  }
}

// Stages a tile's q^P (fields 0..4; FP32: deviations from the element's
// first-node state, with its reference record in refs) and, with_rp, R^P
// (fields 5..9) node-major, [el][p][TS] at X, each value read once.
template <typename T>
__device__ void tau_stage_nm(const TauParams<T>& P, const int32_t* els, int cnt, int nP, bool with_rp, T* X,
                             float* refs) {
  constexpr bool DEV = std::is_same<T, float>::value;
  const MeshView& m = P.m;
  if (DEV)
    for (int el = threadIdx.x; el < cnt; el += blockDim.x)
      tau_ref_make(P.q + 5 * m.off[els[el]], nP, P.gamma64 - 1.0, refs + kTauRefStride * el);
  for (int t = threadIdx.x; t < cnt * nP; t += blockDim.x) {
    const int el = fdiv(t, nP), p = t - el * nP;
    const int64_t o5 = 5 * m.off[els[el]];
    const double* qe = P.q + o5;
    T* x = X + TauTiles<T>::TS * t;
#pragma unroll
    for (int v = 0; v < 5; ++v) x[v] = DEV ? (T)(qe[v * nP + p] - qe[v * nP]) : (T)qe[v * nP + p];
    if (with_rp) {
      if (P.rp) {
#pragma unroll
        for (int v = 0; v < 5; ++v) x[5 + v] = (T)P.rp[o5 + v * nP + p];
      } else {
#pragma unroll
        for (int v = 0; v < 5; ++v) x[5 + v] = P.rp_scratch[o5 + v * nP + p];
      }
    }
  }
  __syncthreads();
}

// Prologue of the isolated Euler sweep, one tile per CTA iteration: the
// isolated R^P of every element into the scratch (unless the caller gave
// R^P), and -1 in the maps for every sweep entry the element's orders
// cannot reach.  Layout: the staged q^P at ST, the fluxes at Ft.
template <typename T, bool AFFINE, bool AXIS, int THREADS>
__global__ void __launch_bounds__(THREADS, (sizeof(T) == 4 ? 1024 : 512) / THREADS) tau_euler_prologue_kernel(
    TauParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  __shared__ float Ref[std::is_same<T, float>::value ? kTauRefElems : 1][kTauRefStride];
  T* sm = reinterpret_cast<T*>(smem_raw);
  constexpr int TS = TauTiles<T>::TS, FS = TauTiles<T>::FS;
  const int S = P.S;
  T* ST = sm;            // [el][p][TS]
  T* Ft = sm + TS * S;   // [el][p][FS]
  const T gm1 = P.gamma - (T)1;
  const MeshView& m = P.m;
  for (int li = blockIdx.x; li < P.n_list; li += gridDim.x) {
    WorkItem w;
    if (!take_item(P.m, P.items, P.ilist[li], P.n_items_all, P.elist, 0, w)) continue;
    if (bad_tile(P.m, w, P.S)) continue;
    const int32_t* els = P.elist + w.first;
    const int cnt = w.count;
    const int P1 = w.n1, P2 = w.n2, P3 = w.n3, n1 = P1 + 1, n2 = P2 + 1, n3 = P3 + 1, nP = n1 * n2 * n3;
    for (int t = threadIdx.x; t < cnt * P.n_sweep; t += blockDim.x) {
      const int el = fdiv(t, P.n_sweep), s = t - el * P.n_sweep;
      if (P.sweep[3 * s] > P1 || P.sweep[3 * s + 1] > P2 || P.sweep[3 * s + 2] > P3) {
        const int64_t idx = (int64_t)els[el] * P.n_sweep + s;
        if (P.map_new) P.map_new[idx] = (T)-1;
        if (P.map_trad) P.map_trad[idx] = (T)-1;
      }
    }
    if (P.rp) continue;
#ifdef DG_BOUNDS_CHECK
    if (std::is_same<T, float>::value && cnt > kTauRefElems) {   // one reference record per element
      if (threadIdx.x == 0) flag_index(P.m);
      continue;
    }
#endif
    tau_stage_nm(P, els, cnt, nP, false, ST, &Ref[0][0]);
    for (int t = threadIdx.x; t < cnt * nP; t += blockDim.x) {
      const int el = fdiv(t, nP), p = t - el * nP;
      const T* met = tile_met<T, AFFINE>(P, els[el], P1, P2, P1, P2, P3);
      T q[5];
#pragma unroll
      for (int v = 0; v < 5; ++v) q[v] = ST[TS * t + v];
      tau_flux_nm<T, AFFINE, AXIS>(gm1, met, nP, p, q, tau_ref_of<T>(&Ref[0][0], el), Ft + FS * t);
    }
    __syncthreads();
    for (int t = threadIdx.x; t < cnt * nP; t += blockDim.x) {
      const int el = fdiv(t, nP), p = t - el * nP;
      const int pj = fdiv(p, n1), k = fdiv(pj, n2), i = p - pj * n1, j = pj - k * n2;
      const int e = els[el];
      const T* met = tile_met<T, AFFINE>(P, e, P1, P2, P1, P2, P3);
      T acc[5];
      tau_div_nm(P.basis, Ft + FS * (el * nP), n1, n2, n3, i, j, k, acc);
      const T iJ = -(T)1 / met_at(met, AFFINE, nP, p, 9);
      const int64_t o5 = 5 * m.off[e];
#pragma unroll
      for (int v = 0; v < 5; ++v) P.rp_scratch[o5 + v * nP + p] = mul_rn(acc[v], iJ);
    }
    __syncthreads();
  }
}

// The isolated Euler sweep, one unit per CTA iteration (a tile and the
// groups (N2, N3) of one N3): q^P and R^P staged once, restricted in xi3 once
// for the unit, in xi2 once per group, then the group's entries in chunks
// (tau_chunk): (1) previous chunk's norms stored, this chunk's slots
// cleared, restriction in xi1 and the fluxes of every coarse node; (2) the
// GL derivative, tau~ = I R^P - R^N and both norms.  Shared memory in S node
// slots of TS, FS or RS values: A3, A2, then Ft and A1, with the staged tile
// ST over Ft and A1 (it is read only by the xi3 pass, before them); compact
// (units of one group): A3 and then A1, ST and then A2, Ft.  Every region
// starts at an even float, as the packed FP32 loads need.
template <typename T, bool AFFINE, bool AXIS, int THREADS>
__global__ void __launch_bounds__(THREADS, (sizeof(T) == 4 ? 1024 : 512) / THREADS) tau_euler_kernel(TauParams<T> P) {
  extern __shared__ __align__(16) unsigned char smem_raw[];
  T* sm = reinterpret_cast<T*>(smem_raw);
  typedef typename Bits<T>::type B;
  __shared__ B na2[2][kVolThreads], nb2[2][kVolThreads];   // per-element norms, two chunks in flight
  __shared__ float Ref[std::is_same<T, float>::value ? kTauRefElems : 1][kTauRefStride];
  __shared__ int4 gtab[kTauBatchGroups];    // a batch's groups: N2 + 1, A2 offset and size (nodes)
  __shared__ int4 etab[kTauBatchEntries];   // its entries: sweep index, N1, N2 + 1, A2 offset
  __shared__ int btab[4];                   // groups in the batch, entries in etab, next group and entry
  constexpr int TS = TauTiles<T>::TS, FS = TauTiles<T>::FS, RS = TauTiles<T>::RS;
  const int S = P.S;
  T* A3 = sm;
  T* A2 = sm + TS * S;
  T* Ft = sm + 2 * TS * S;
  T* A1 = P.compact ? sm : Ft + FS * S;
  T* ST = P.compact ? A2 : Ft;
  const MeshView& m = P.m;
  const T gm1 = P.gamma - (T)1;
  for (int ui = blockIdx.x; ui < P.n_list; ui += gridDim.x) {
    const int4 u = P.units[ui];
    WorkItem w;
    if (!take_item(P.m, P.items, u.x, P.n_items_all, P.elist, 0, w)) continue;
    if (bad_tile(P.m, w, P.S) || bad_group(P, w, u.y)) continue;
#ifdef DG_BOUNDS_CHECK
    // one norm slot per element and chunk entry; one reference record per
    // element (FP32); the compact layout holds one group
    if (w.count > kVolThreads || (std::is_same<T, float>::value && w.count > kTauRefElems) ||
        (P.compact && u.z != 1)) {
      if (threadIdx.x == 0) flag_index(P.m);
      continue;
    }
#endif
    const int32_t* els = P.elist + w.first;
    const int cnt = w.count;
    const int P1 = w.n1, P2 = w.n2, P3 = w.n3, n1 = P1 + 1, n2 = P2 + 1, n3 = P3 + 1, nP = n1 * n2 * n3;
    const int N3 = P.groups[u.y].y, c3 = N3 + 1, n12 = n1 * n2;
#ifdef DG_BOUNDS_CHECK
    {  // every group of the unit: inside the group list, orders within the tile's, entries inside the sweep, one N3
      bool bad = false;
      for (int gi = u.y + 1; gi < u.y + u.z && !bad; ++gi) {
        bad = bad_group(P, w, gi);
        if (!bad && P.groups[gi].y != N3) {
          if (threadIdx.x == 0) flag_index(m);
          bad = true;
        }
      }
      if (bad) continue;
    }
#endif
    tau_stage_nm(P, els, cnt, nP, true, ST, &Ref[0][0]);
    {  // xi3, once for the unit's groups: A3[el][i + n1 (j + n2 k)]
      const T* I3 = P.basis + c_boff.I[P3][N3];
      const int per = n12 * c3;
      for (int t = threadIdx.x; t < cnt * per; t += blockDim.x) {
        const int el = fdiv(t, per), x = t - el * per, k = fdiv(x, n12), ij = x - k * n12;
        T acc[10];
        restrict_node(n3, I3 + k * n3, ST + TS * (el * nP + ij), TS * n12, acc);
        T* o = A3 + TS * t;
#pragma unroll
        for (int c = 0; c < 10; ++c) o[c] = acc[c];
      }
      __syncthreads();
    }
    // The groups of this N3 run in batches whose xi2-restricted tiles fit the
    // S node slots of A2 together (the compact layout: one group), and the
    // chunks of a batch draw on the entries of all its groups: a small group
    // alone would leave most of the CTA idle in its passes.  Thread 0 lays
    // out the batch (gtab) and its entries within the tile's orders (etab,
    // in pieces of at most kTauBatchEntries); every other value below is the
    // same in every thread.
    for (int gb = u.y; gb < u.y + u.z;) {
      if (threadIdx.x == 0) {
        int ge = gb, used = 0;
        while (ge < u.y + u.z && ge - gb < kTauBatchGroups) {
          const int c2 = P.groups[ge].x + 1, sz = cnt * n1 * c2 * c3;
          if (ge > gb && (P.compact || used + sz > S)) break;
          gtab[ge - gb] = make_int4(c2, used, sz, 0);
          used += sz;
          ++ge;
        }
        btab[0] = ge - gb;
        btab[2] = 0;   // next group and entry of the batch's entry table
        btab[3] = 0;
        tau_fill_entries(P, gb, ge - gb, P1, gtab, etab, btab);
      }
      __syncthreads();
      const int nb = btab[0];
      const int pin = n12 * c3;
      {  // xi2 for every group of the batch: A2[gtab.y + el per2 + i + n1 (j' + c2 k')]
        const int4 gl = gtab[nb - 1];
        const int tot = gl.y + gl.z;
        for (int t = threadIdx.x; t < tot; t += blockDim.x) {
          int b = 0;
          while (b + 1 < nb && t >= gtab[b + 1].y) ++b;
          const int4 gg = gtab[b];
          const int c2 = gg.x, per2 = n1 * c2 * c3, tt = t - gg.y;
          const int el = fdiv(tt, per2), x = tt - el * per2, xj = fdiv(x, n1), k = fdiv(xj, c2), i = x - xj * n1,
                    j = xj - k * c2;
          T acc[10];
          restrict_node(n2, P.basis + c_boff.I[P2][c2 - 1] + j * n2, A3 + TS * (el * pin + i + n12 * k), TS * n1,
                        acc);
          T* o = A2 + TS * t;
#pragma unroll
          for (int c = 0; c < 10; ++c) o[c] = acc[c];
        }
        __syncthreads();
      }
      const T* w3 = P.basis + c_boff.W[N3];
      for (;;) {   // the pieces of the batch's entry table
        const int n_tab = btab[1], next_g = btab[2];
        int prev_first = 0, prev_k = 0, buf = 0;
        for (int first = 0; first < n_tab;) {
          int total;
          const int k = tau_batch_chunk(etab, first, n_tab, cnt, c3, S, total);
          const int nsl = (prev_k > k ? prev_k : k) * cnt;
          for (int sl = threadIdx.x; sl < nsl; sl += blockDim.x) {
            const int j = fdiv(sl, cnt), el = sl - j * cnt;
            if (j < prev_k) {
              const int64_t idx = (int64_t)els[el] * P.n_sweep + etab[prev_first + j].x;
              map_store(P.map_new, idx, P.accumulate, Bits<T>::val(na2[buf ^ 1][sl]));
              map_store(P.map_trad, idx, P.accumulate, Bits<T>::val(nb2[buf ^ 1][sl]));
            }
            if (j < k) {
              na2[buf][sl] = 0;
              nb2[buf][sl] = 0;
            }
          }
          // (1) xi1 restriction and the fluxes of every coarse node of the chunk
          for (int t = threadIdx.x; t < total; t += blockDim.x) {
            int base, j;
            const int4 en = tau_batch_item(etab, first, t, cnt, c3, base, j);
            const int M1 = en.y, c1 = M1 + 1, c2 = en.z, nN = c1 * c2 * c3, tt = t - base;
            const int el = fdiv(tt, nN), x = tt - el * nN, jk = fdiv(x, c1), i = x - jk * c1;
            T acc[10];
            restrict_node(n1, P.basis + c_boff.I[P1][M1] + i * n1, A2 + TS * (en.w + el * (n1 * c2 * c3) + n1 * jk),
                          TS, acc);
            const T* met = tile_met<T, AFFINE>(P, els[el], P1, P2, M1, c2 - 1, N3);
            tau_flux_nm<T, AFFINE, AXIS>(gm1, met, nN, x, acc, tau_ref_of<T>(&Ref[0][0], el), Ft + FS * t);
            T* o = A1 + RS * t;
#pragma unroll
            for (int v = 0; v < 5; ++v) o[v] = acc[5 + v];    // I R^P
          }
          __syncthreads();
          // (2) derivative, tau~ and both norms (whole warps, for the norms' warp reduction)
          for (int t0 = threadIdx.x & ~31; t0 < total; t0 += blockDim.x) {
            const int t = t0 + (threadIdx.x & 31);
            int slot = -1;
            T a = 0, b = 0;
            if (t < total) {
              int base, j;
              const int4 en = tau_batch_item(etab, first, t, cnt, c3, base, j);
              const int M1 = en.y, c1 = M1 + 1, c2 = en.z, nN = c1 * c2 * c3, tt = t - base;
              const int el = fdiv(tt, nN), p = tt - el * nN, pj = fdiv(p, c1), kk = fdiv(pj, c2), i = p - pj * c1,
                        jj = pj - kk * c2;
              const T* met = tile_met<T, AFFINE>(P, els[el], P1, P2, M1, c2 - 1, N3);
              T acc[5];
              tau_div_nm(P.basis, Ft + FS * (base + el * nN), c1, c2, c3, i, jj, kk, acc);
              const T J = met_at(met, AFFINE, nN, p, 9);
              const T iJ = -(T)1 / J;
              const T Jw = J * P.basis[c_boff.W[M1] + i] * P.basis[c_boff.W[c2 - 1] + jj] * w3[kk];
              const T* ir = A1 + RS * t;
#pragma unroll
              for (int v = 0; v < 5; ++v) {
                const T d = ir[v] - mul_rn(acc[v], iJ);   // tau~ = I R^P - R^N(I q^P)
                a = tmax(a, (T)fabs(d));
                b = tmax(b, (T)fabs(Jw * d));
              }
              slot = j * cnt + el;
            }
            warp_norm_max(na2[buf], nb2[buf], slot, a, b);
          }
          __syncthreads();
          prev_first = first;
          prev_k = k;
          buf ^= 1;
          first += k;
        }
        for (int sl = threadIdx.x; sl < prev_k * cnt; sl += blockDim.x) {
          const int j = fdiv(sl, cnt), el = sl - j * cnt;
          const int64_t idx = (int64_t)els[el] * P.n_sweep + etab[prev_first + j].x;
          map_store(P.map_new, idx, P.accumulate, Bits<T>::val(na2[buf ^ 1][sl]));
          map_store(P.map_trad, idx, P.accumulate, Bits<T>::val(nb2[buf ^ 1][sl]));
        }
        __syncthreads();   // the tables and norm slots are free again
        if (next_g >= nb) break;
        if (threadIdx.x == 0) tau_fill_entries(P, gb, nb, P1, gtab, etab, btab);
        __syncthreads();
      }
      gb += nb;
    }   // batches of groups
  }
}

// Non-isolated tau, final step for one sweep entry s of orders N: per
// element with N <= P, tau~ = I_{N<-P} R^P - R_c (R_c the residual of the
// coarse discretisation), both norms.  Coarse J from the coarse mesh.
template <typename MT, bool AFFINE>
__global__ void __launch_bounds__(kTauThreads) tau_combine_kernel(MeshView fine, MeshView coarse, const double* rp,
                                                                  const double* rc, const double* basis, int N1,
                                                                  int N2, int N3, int s, int n_sweep, int S,
                                                                  int accumulate, MT* map_new, MT* map_trad,
                                                                  int n_elem) {
  extern __shared__ double smd[];
  __shared__ double red[2][kTauThreads / 32];
  double* B0 = smd;
  double* B1 = B0 + 5 * S;
  double* B2 = B1 + 5 * S;
  for (int e = blockIdx.x; e < n_elem; e += gridDim.x) {
    int n1, n2, n3;
    orders_of(fine, e, n1, n2, n3);
    const int64_t idx = (int64_t)e * n_sweep + s;
    if (N1 > n1 - 1 || N2 > n2 - 1 || N3 > n3 - 1) {
      if (threadIdx.x == 0) {
        if (map_new) map_new[idx] = (MT)-1;
        if (map_trad) map_trad[idx] = (MT)-1;
      }
      continue;
    }
    const int nP = n1 * n2 * n3;
    const int64_t o = fine.off[e], oc = coarse.off[e];
    for (int p = threadIdx.x; p < nP; p += blockDim.x)
      for (int v = 0; v < 5; ++v) B0[v * S + p] = rp[5 * o + v * nP + p];
    __syncthreads();
    apply_dir_tile(basis + c_boff.I[n3 - 1][N3], N3 + 1, n3, 2, n1, n2, n3, B0, S, B1, S, 5);
    apply_dir_tile(basis + c_boff.I[n2 - 1][N2], N2 + 1, n2, 1, n1, n2, N3 + 1, B1, S, B2, S, 5);
    apply_dir_tile(basis + c_boff.I[n1 - 1][N1], N1 + 1, n1, 0, n1, N2 + 1, N3 + 1, B2, S, B0, S, 5);
    const int c1 = N1 + 1, c2 = N2 + 1, c3 = N3 + 1, nN = c1 * c2 * c3;
    const double* w1 = basis + c_boff.W[N1];
    const double* w2 = basis + c_boff.W[N2];
    const double* w3 = basis + c_boff.W[N3];
    double a = 0, b = 0;
    for (int p = threadIdx.x; p < nN; p += blockDim.x) {
      const int i = p % c1, j = (p / c1) % c2, k = p / (c1 * c2);
      double J = metric<AFFINE>(coarse.metric, e, oc, nN, p, 9);
      double Jw = J * w1[i] * w2[j] * w3[k];
      for (int v = 0; v < 5; ++v) {
        double t = B0[v * S + p] - rc[5 * oc + v * nN + p];
        a = fmax(a, fabs(t));
        b = fmax(b, fabs(Jw * t));
      }
    }
    block_max2(a, b, red);
    if (threadIdx.x == 0) {
      if (map_new) map_new[idx] = accumulate ? (MT)fmax((double)map_new[idx], a) : (MT)a;
      if (map_trad) map_trad[idx] = accumulate ? (MT)fmax((double)map_trad[idx], b) : (MT)b;
    }
    __syncthreads();
  }
}

// Per-element projection of the state between orders: mode 0 (set_orders):
// interpolation where the order rises, L2 projection where it falls;
// mode 1 (restriction): interpolation in every direction.
__global__ void __launch_bounds__(kTauThreads) project_kernel(const int32_t* ord_old, const int64_t* off_old,
                                                              const int32_t* ord_new, const int64_t* off_new,
                                                              const double* basis, const double* q_old,
                                                              double* q_new, int n_elem, int S, int mode) {
  extern __shared__ double smd[];
  double* B0 = smd;
  double* B1 = B0 + 5 * S;
  for (int e = blockIdx.x; e < n_elem; e += gridDim.x) {
    int f[3], t[3];
    for (int d = 0; d < 3; ++d) {
      f[d] = ord_old[3 * e + d];
      t[d] = ord_new[3 * e + d];
    }
    const int nf = (f[0] + 1) * (f[1] + 1) * (f[2] + 1), nt = (t[0] + 1) * (t[1] + 1) * (t[2] + 1);
    for (int p = threadIdx.x; p < nf; p += blockDim.x)
      for (int v = 0; v < 5; ++v) B0[v * S + p] = q_old[5 * off_old[e] + v * nf + p];
    __syncthreads();
    int ext[3] = {f[0] + 1, f[1] + 1, f[2] + 1};
    double* src = B0;
    double* dst = B1;
    for (int d = 0; d < 3; ++d) {
      int mo = (mode == 1 || t[d] >= f[d]) ? c_boff.I[f[d]][t[d]] : c_boff.P[f[d]][t[d]];
      apply_dir_tile(basis + mo, t[d] + 1, f[d] + 1, d, ext[0], ext[1], ext[2], src, S, dst, S, 5);
      ext[d] = t[d] + 1;
      double* tmp = src;
      src = dst;
      dst = tmp;
    }
    for (int p = threadIdx.x; p < nt; p += blockDim.x)
      for (int v = 0; v < 5; ++v) q_new[5 * off_new[e] + v * nt + p] = src[v * S + p];
    __syncthreads();
  }
}

MeshView view(const dg_mesh_impl* m);

FaceParams dgk_face_params_for(dg_mesh_impl* m, const double* q, double* surf);
VolParams dgk_vol_params_for(dg_mesh_impl* m, const double* q, const double* surf, double* r);

MeshView view(const dg_mesh_impl* m) {
  MeshView v;
  v.ord = m->d_ord;
  v.off = m->d_off;
  v.soff = m->d_soff;
  v.metric = m->d_metric;
  v.ph = m->phys;
  v.n_elem = m->n_elem;
  v.n_nodes = m->n_nodes;
  v.n_surf = m->h_soff.empty() ? 0 : m->h_soff[m->n_elem];
  v.err = m->d_err;
  return v;
}

int grid_for(int work, int per_sm_blocks) {
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  int cap = sms * per_sm_blocks;
  return work < cap ? (work > 0 ? work : 1) : cap;
}

// Raise a kernel's dynamic shared-memory limit to the device opt-in maximum
// minus its static shared memory, once per kernel and device (so that no
// attribute call is needed later, e.g. under stream capture).  Done for any
// dynamic size: the default limit of 48 KB covers static + dynamic.
template <typename K>
cudaError_t allow_smem(K kernel, size_t bytes) {
  static std::map<std::pair<int, const void*>, int> raised;   // (device, kernel) -> limit set
  if (bytes == 0) return cudaSuccess;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  auto key = std::make_pair(dev, reinterpret_cast<const void*>(kernel));
  auto it = raised.find(key);
  if (it != raised.end() && (int)bytes <= it->second) return cudaSuccess;
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  cudaError_t e = cudaFuncGetAttributes(&fa, kernel);
  if (e) return e;
  const int limit = optin - (int)fa.sharedSizeBytes;   // dynamic + static <= opt-in maximum
  if ((int)bytes > limit) return cudaErrorInvalidValue;
  e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, limit);
  if (e == cudaSuccess) raised[key] = limit;
  return e;
}

// brackets a launch with the mesh's timing/counting hooks
struct Prof {
  dg_mesh_impl* m;
  int id;
  Prof(dg_mesh_impl* mm, int k, int n = 1) : m(mm), id(k) { dg_prof_begin(m, k, n); }
  ~Prof() { dg_prof_end(m, id); }
};

FaceParams dgk_face_params_for(dg_mesh_impl* m, const double* q, double* surf) {
  FaceParams P;
  P.m = view(m);
  P.faces = m->d_faces;
  P.n_faces = m->n_faces;
  P.q = q;
  P.grad = nullptr;
  P.surf = surf;
  P.basis = m->basis64;
  P.np_max = m->max_order + 1;
  P.warp_smem = 25 * P.np_max * P.np_max;
  P.fnodes = reinterpret_cast<const int2*>(m->d_fnodes);
  P.n_fnodes = m->n_fnodes;
  return P;
}

VolParams dgk_vol_params_for(dg_mesh_impl* m, const double* q, const double* surf, double* r) {
  VolParams P;
  memset(&P, 0, sizeof(P));
  P.m = view(m);
  P.items = m->d_vitems;
  P.n_items = m->n_vitems;
  P.n_items_all = m->n_vitems;
  P.elist = m->d_velist;
  P.q = q;
  P.surf = surf;
  P.basis = m->basis64;
  P.out = r;
  P.err = m->d_err;
  return P;
}

template <bool AFF, bool AX, bool NSV>
cudaError_t launch_face(dg_mesh_impl* m, const FaceParams& P, size_t smem, int grid) {
  (void)smem;
  (void)grid;
  if (P.n_fnodes == 0) return cudaSuccess;
  const int blocks = (P.n_fnodes + kFaceNodeThreads - 1) / kFaceNodeThreads;
  face_node_flux_kernel<AFF, AX, NSV><<<blocks, kFaceNodeThreads, 0, m->stream>>>(P);
  return cudaGetLastError();
}

cudaError_t dispatch_face(dg_mesh_impl* m, const FaceParams& P, size_t smem, int grid) {
  const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
  if (m->axis) return ns ? launch_face<true, true, true>(m, P, smem, grid) : launch_face<true, true, false>(m, P, smem, grid);
  if (m->affine)
    return ns ? launch_face<true, false, true>(m, P, smem, grid) : launch_face<true, false, false>(m, P, smem, grid);
  return ns ? launch_face<false, false, true>(m, P, smem, grid) : launch_face<false, false, false>(m, P, smem, grid);
}

template <bool AFF, bool AX, bool NSV>
cudaError_t launch_volume(dg_mesh_impl* m, const VolParams& P, size_t smem, int grid) {
  // Tiles whose shared memory admits two CTAs per SM (401-700 nodes, 20
  // doubles a node) run 384 threads and those admitting one (more than 700
  // nodes) 768, so that every class keeps about 24 warps per SM to feed the
  // FP64 pipe (8 a CTA of 256 threads otherwise).
  cudaError_t err;
  if (smem > kVolTwoCtaBytes) {
    if ((err = allow_smem(volume_kernel<AFF, AX, NSV, 3 * kVolThreads>, smem))) return err;
    volume_kernel<AFF, AX, NSV, 3 * kVolThreads><<<grid, 3 * kVolThreads, smem, m->stream>>>(P);
  } else if (smem > kVolThreeCtaBytes) {
    if ((err = allow_smem(volume_kernel<AFF, AX, NSV, 3 * kVolThreads / 2>, smem))) return err;
    volume_kernel<AFF, AX, NSV, 3 * kVolThreads / 2><<<grid, 3 * kVolThreads / 2, smem, m->stream>>>(P);
  } else {
    if ((err = allow_smem(volume_kernel<AFF, AX, NSV, kVolThreads>, smem))) return err;
    volume_kernel<AFF, AX, NSV, kVolThreads><<<grid, kVolThreads, smem, m->stream>>>(P);
  }
  return cudaGetLastError();
}

cudaError_t dispatch_volume_one(dg_mesh_impl* m, const VolParams& P, size_t smem, int grid) {
  const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
  if (m->axis)
    return ns ? launch_volume<true, true, true>(m, P, smem, grid) : launch_volume<true, true, false>(m, P, smem, grid);
  if (m->affine)
    return ns ? launch_volume<true, false, true>(m, P, smem, grid) : launch_volume<true, false, false>(m, P, smem, grid);
  return ns ? launch_volume<false, false, true>(m, P, smem, grid) : launch_volume<false, false, false>(m, P, smem, grid);
}

// Every numerical face flux into the face buffer surf: conforming and
// boundary faces one warp each, p-nonconforming faces in shape batches.
cudaError_t launch_all_faces(dg_mesh_impl* m, const double* q, const double* grad, double* surf,
                             const double* trace = nullptr) {
  cudaError_t err;
  if (m->n_faces) {
    FaceParams P = dgk_face_params_for(m, q, surf);
    P.grad = grad;
    const int grid = (m->n_faces + kFaceWarps - 1) / kFaceWarps;
    Prof pr(m, DG_KERNEL_FACE_FLUX);
    if ((err = dispatch_face(m, P, 0, grid))) return err;
  }
  if (m->n_mbatches) {
    Prof pr(m, DG_KERNEL_MORTAR);
    MortarParams M{};
    M.m = view(m);
    M.batches = reinterpret_cast<const MortarBatch*>(m->d_mbatches);
    M.n_batches = m->n_mbatches;
    M.n_mfaces = m->n_mfaces;
    M.faces = m->d_mfaces;
    M.q = q;
    M.surf = surf;
    M.basis = m->basis64;
    M.grad = grad;
    M.trace = m->general_mortars ? nullptr : trace;
    const size_t smem = sizeof(double) * m->mortar_smem;
    const int grid = m->n_mbatches;   // one CTA per batch, largest first
    if (m->general_mortars) {
      const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
#define DG_GMORTAR(AFF, MODE)                                                       \
  {                                                                                 \
    if ((err = allow_smem(mortar_general_kernel<AFF, MODE>, smem))) return err;     \
    mortar_general_kernel<AFF, MODE><<<grid, kVolThreads, smem, m->stream>>>(M);    \
  }
      if (m->affine) {
        if (ns) DG_GMORTAR(true, 1) else DG_GMORTAR(true, 0)
      } else {
        if (ns) DG_GMORTAR(false, 1) else DG_GMORTAR(false, 0)
      }
    } else if (m->axis) {
      if ((err = allow_smem(mortar_kernel<true>, smem))) return err;
      mortar_kernel<true><<<grid, kVolThreads, smem, m->stream>>>(M);
    } else {
      if ((err = allow_smem(mortar_kernel<false>, smem))) return err;
      mortar_kernel<false><<<grid, kVolThreads, smem, m->stream>>>(M);
    }
    if ((err = cudaGetLastError())) return err;
  }
  return cudaSuccess;
}

size_t mortar_smem_doubles(int count, int la, int lb, int ra, int rb) {
  MortarBatch B{0, count, la, lb, ra, rb};
  return mortar_batch_smem(B);
}

// The volume kernel once per volume class (tiles up to kVolSplitNodes nodes,
// and the larger ones), each launch with the shared memory of its largest
// tile (20 doubles per node), so that a few large elements do not lower the
// occupancy of all the others.
cudaError_t dispatch_volume(dg_mesh_impl* m, const VolParams& P0, size_t, int) {
  cudaError_t err;
  for (auto& c : m->vol_classes) {
    VolParams P = P0;
    P.ilist = c.d_list;
    P.n_items = c.n;
    if ((err = dispatch_volume_one(m, P, sizeof(double) * 20 * c.S, c.n))) return err;   // one CTA per tile
  }
  return cudaSuccess;
}

}  // namespace

size_t dg_mortar_smem_doubles(int count, int la, int lb, int ra, int rb) {
  return mortar_smem_doubles(count, la, lb, ra, rb);
}

size_t dg_mortar_general_smem_doubles(int count, int la, int lb, int ra, int rb, bool ns) {
  const MortarBatch B{0, count, la, lb, ra, rb};
  return ns ? std::max(mortar_general_smem<1>(B), mortar_general_smem<2>(B)) : mortar_general_smem<0>(B);
}

namespace dgk {

void upload_basis(int device, const BasisOffsets& off, const std::vector<double>& data, const double** d64,
                  const float** d32) {
  (void)device;
  cudaMemcpyToSymbol(c_boff, &off, sizeof(off));
  std::vector<uint2> fd(kFdivMax + 1, make_uint2(0u, 0u));
  for (int d = 1; d <= kFdivMax; ++d) {
    uint32_t l = 0;
    while ((1u << l) < (uint32_t)d) ++l;
    const uint64_t mm = ((uint64_t(1) << 32) * ((uint64_t(1) << l) - (uint64_t)d)) / (uint64_t)d + 1;
    fd[d] = make_uint2((uint32_t)mm, l);
  }
  cudaMemcpyToSymbol(c_fdiv, fd.data(), sizeof(uint2) * fd.size());
  double* a = nullptr;
  float* b = nullptr;
  cudaMalloc(&a, sizeof(double) * data.size());
  cudaMalloc(&b, sizeof(float) * data.size());
  cudaMemcpy(a, data.data(), sizeof(double) * data.size(), cudaMemcpyHostToDevice);
  std::vector<float> f(data.begin(), data.end());
  cudaMemcpy(b, f.data(), sizeof(float) * f.size(), cudaMemcpyHostToDevice);
  *d64 = a;
  *d32 = b;
}

static FaceParams face_params(dg_mesh_impl* m, const double* q, const double* grad) {
  FaceParams P;
  P.m = view(m);
  P.faces = m->d_faces;
  P.n_faces = m->n_faces;
  P.q = q;
  P.grad = grad;
  P.surf = m->d_surf;
  P.basis = m->basis64;
  P.np_max = m->max_order + 1;
  P.warp_smem = 25 * P.np_max * P.np_max;
  P.fnodes = reinterpret_cast<const int2*>(m->d_fnodes);
  P.n_fnodes = m->n_fnodes;
  return P;
}

cudaError_t face_flux(dg_mesh_impl* m, const double* q, const double* grad, bool isolated) {
  (void)isolated;
  return launch_all_faces(m, q, grad, m->d_surf);
}

cudaError_t face_flux_rk(dg_mesh_impl* m, const double* q, bool trace_valid) {
  return launch_all_faces(m, q, m->d_grad, m->d_surf, trace_valid ? m->d_trace : nullptr);
}

cudaError_t face_qhat(dg_mesh_impl* m, const double* q) {
  cudaError_t err;
  Prof pr(m, DG_KERNEL_FACE_QHAT);
  if (m->n_faces) {
    FaceParams P = face_params(m, q, nullptr);
    int grid = (m->n_faces + kFaceWarps - 1) / kFaceWarps;
    if (m->affine) face_qhat_kernel<true><<<grid, 32 * kFaceWarps, 0, m->stream>>>(P, m->d_surfq);
    else face_qhat_kernel<false><<<grid, 32 * kFaceWarps, 0, m->stream>>>(P, m->d_surfq);
    if ((err = cudaGetLastError())) return err;
  }
  if (m->n_mbatches && m->general_mortars) {   // BR1 q-hat on the mortars
    MortarParams M{};
    M.m = view(m);
    M.batches = reinterpret_cast<const MortarBatch*>(m->d_mbatches);
    M.n_batches = m->n_mbatches;
    M.n_mfaces = m->n_mfaces;
    M.faces = m->d_mfaces;
    M.q = q;
    M.surf = m->d_surfq;
    M.basis = m->basis64;
    M.grad = nullptr;
    const size_t smem = sizeof(double) * m->mortar_smem;
    const int grid = m->n_mbatches;
    if (m->affine) DG_GMORTAR(true, 2) else DG_GMORTAR(false, 2)
    if ((err = cudaGetLastError())) return err;
  }
  return cudaSuccess;
}
#undef DG_GMORTAR

static VolParams vol_params(dg_mesh_impl* m, const double* q) {
  VolParams P;
  memset(&P, 0, sizeof(P));
  P.m = view(m);
  P.items = m->d_vitems;
  P.n_items = m->n_vitems;
  P.n_items_all = m->n_vitems;
  P.elist = m->d_velist;
  P.q = q;
  P.grad = m->d_grad;
  P.surf = m->d_surf;
  P.surfq = m->d_surfq;
  P.basis = m->basis64;
  P.err = m->d_err;
  return P;
}

cudaError_t gradient(dg_mesh_impl* m, const double* q, double* grad, bool isolated) {
  VolParams P = vol_params(m, q);
  P.out = grad;
  P.isolated = isolated;
  cudaError_t err;
  Prof pr(m, DG_KERNEL_GRADIENT, (int)m->vol_classes.size());
  for (auto& c : m->vol_classes) {   // one launch per tile-size class (15 doubles per node)
    P.ilist = c.d_list;
    P.n_items = c.n;
    const size_t smem = sizeof(double) * 15 * c.S;
    const int grid = grid_for(c.n, 8);
    if (m->affine) {
      if ((err = allow_smem(gradient_kernel<true>, smem))) return err;
      gradient_kernel<true><<<grid, kVolThreads, smem, m->stream>>>(P);
    } else {
      if ((err = allow_smem(gradient_kernel<false>, smem))) return err;
      gradient_kernel<false><<<grid, kVolThreads, smem, m->stream>>>(P);
    }
    if ((err = cudaGetLastError())) return err;
  }
  return cudaSuccess;
}

cudaError_t volume(dg_mesh_impl* m, const double* q, const double* grad, double* r, bool isolated, int rk_stage,
                   double* q_io, double* g_io, const double* dt_dev) {
  static const double A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
  static const double B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
  VolParams P = vol_params(m, q);
  P.grad = grad;
  P.out = r;
  P.isolated = isolated;
  if (rk_stage >= 0) {
    P.rk = 1;
    P.rk_first = rk_stage == 0;
    P.rkA = A[rk_stage];
    P.rkB = B[rk_stage];
    P.q_io = q_io;
    P.g_io = g_io;
    P.dt = dt_dev;
    P.trace_out = q_io == q ? m->d_trace : nullptr;   // the stepped state's traces (dg_rk_step's own q)
  }
  Prof pr(m, DG_KERNEL_VOLUME, (int)m->vol_classes.size());
  return dispatch_volume(m, P, 0, 0);
}

// bits: the FP64 maximum (bits[0]); bits[1] holds the FP32 filter maximum
cudaError_t max_dt_bits(dg_mesh_impl* m, const double* q, unsigned long long* bits) {
  VolParams P = vol_params(m, q);
  cudaError_t err = cudaMemsetAsync(bits, 0, 2 * sizeof(unsigned long long), m->stream);
  if (err) return err;
  unsigned* m32 = reinterpret_cast<unsigned*>(bits + 1);
  const DevPhys& ph = P.m.ph;
  const double gpr = ph.gamma / ph.Pr > 1.0 ? ph.gamma / ph.Pr : 1.0;
  P.k64 = ScaleConst<double>{ph.gamma - 1.0, ph.gamma, ph.mu, gpr, ph.eqs == DG_NAVIER_STOKES};
  P.k32 = ScaleConst<float>{(float)(ph.gamma - 1.0), (float)ph.gamma, (float)ph.mu, (float)gpr, P.k64.ns};
  P.metric32 = m->d_metric32;
  int grid = grid_for(m->n_vitems, 8);
  Prof pr(m, DG_KERNEL_MAX_DT, 2);
  if (m->axis) {
    dt_filter_kernel<true, true><<<grid, kVolThreads, 0, m->stream>>>(P, m32);
    dt_kernel<true, true><<<grid, kVolThreads, 0, m->stream>>>(P, m32, bits);
  } else if (m->affine) {
    dt_filter_kernel<true, false><<<grid, kVolThreads, 0, m->stream>>>(P, m32);
    dt_kernel<true, false><<<grid, kVolThreads, 0, m->stream>>>(P, m32, bits);
  } else {
    dt_filter_kernel<false, false><<<grid, kVolThreads, 0, m->stream>>>(P, m32);
    dt_kernel<false, false><<<grid, kVolThreads, 0, m->stream>>>(P, m32, bits);
  }
  return cudaGetLastError();
}

cudaError_t max_dt(dg_mesh_impl* m, const double* q, double cfl, double* dt_dev) {
  unsigned long long* bits = reinterpret_cast<unsigned long long*>(m->d_scratch);
  cudaError_t err = max_dt_bits(m, q, bits);
  if (err) return err;
  Prof pr(m, DG_KERNEL_MAX_DT, 1);
  dt_finalize<<<1, 1, 0, m->stream>>>(bits, cfl, dt_dev);
  return cudaGetLastError();
}

// Dynamic shared memory of the isolated sweep for a class of elements with at
// most S nodes: restriction buffers A3, A2, A1 / staging (10 S each) and
// fluxes (15 S), plus the BR1 gradient (15 S) for Navier-Stokes; the compact
// layout (units of one group) needs 10 S less of the restriction buffers and
// A1 within A3's place.
size_t tau_smem_for(int S, bool ns, bool fp32, bool compact) {
  // Euler: node-major tiles, A3 and A2 (TS values a node slot each), A1 (RS)
  // and Ft (FS); the compact layout has A1 inside A3's place
  const int TS = fp32 ? TauTiles<float>::TS : TauTiles<double>::TS;
  const int FS = fp32 ? TauTiles<float>::FS : TauTiles<double>::FS;
  const int fields = ns ? (compact ? 50 : 60) : (compact ? 2 * TS + FS : 2 * TS + TauTiles<float>::RS + FS);
  return (size_t)fields * S * (fp32 ? sizeof(float) : sizeof(double));
}

// Static shared memory of the sweep kernel: the double-buffered norm slots,
// the FP32 reference records, and the bytes the compiler may add.
size_t tau_static_bytes(bool fp32) {
  return 2 * 2 * kVolThreads * (fp32 ? sizeof(unsigned) : sizeof(unsigned long long)) +
         (fp32 ? kTauRefElems : 1) * kTauRefStride * sizeof(float) +
         (kTauBatchGroups + kTauBatchEntries) * sizeof(int4) + 256;
}

// The compact layout where the other does not fit the device.
bool tau_use_compact(int S, bool ns, bool fp32, int limit) {
  return tau_smem_for(S, ns, fp32, false) + tau_static_bytes(fp32) > (size_t)limit;
}

// CTA size of the Euler sweep for a CTA of `bytes` of shared memory: 256
// threads while three or more fit an SM, 512 for two, 1024 for one (FP32);
// FP64 at up to 128 registers a thread stops at 512.  (Measured: 512 threads
// in a class that fits three 256-thread CTAs ran 2% slower; a class of one
// or two CTAs per SM ran 8% faster on the 48^3 mesh with orders 2-8.)
int tau_euler_threads(size_t bytes, bool fp32) {
  const size_t sm_bytes = 228 * 1024;
  const int ctas = (int)(sm_bytes / (bytes + 1024));
  const int t = ctas >= 3 ? 256 : (ctas == 2 ? 512 : 1024);
  return fp32 ? t : (t > 512 ? 512 : t);
}

size_t tau_smem_bytes(dg_mesh_impl* m, bool fp32, int limit) {
  size_t mx = 0;
  const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
  for (auto& c : m->tau_classes)
    mx = std::max(mx, tau_smem_for(c.S, ns, fp32, tau_use_compact(c.S, ns, fp32, limit)) + tau_static_bytes(fp32));
  return mx;
}

template <typename T>
static cudaError_t tau_launch(dg_mesh_impl* m, TauParams<T> P, bool fp32) {
  const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
  cudaError_t err;
  Prof pr(m, DG_KERNEL_TAU, 2 * (int)m->tau_classes.size());
  P.items = m->d_items;
  P.n_items_all = m->n_items;
  P.n_groups = m->n_tgroups;
  P.n_gentries = m->n_tgentries;
  P.elist = m->d_elist;
  P.groups = reinterpret_cast<const int4*>(m->d_tgroups);
  P.gentries = reinterpret_cast<const int2*>(m->d_tgentries);
  int limit = 0;
  if ((err = cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device))) return err;
  m->tau_last_units.assign(m->tau_classes.size(), 0);
  m->tau_last_shared.assign(m->tau_classes.size(), 0);
  // prologue over every class first, then the sweep units of every class
  for (int phase = 0; phase < 2; ++phase) {
    for (size_t k = 0; k < m->tau_classes.size(); ++k) {
      const auto& c = m->tau_classes[k];
      const bool compact = tau_use_compact(c.S, ns, fp32, limit);   // then units of one group each
      P.S = c.S;
      P.compact = compact;
      P.ilist = c.d_list;
      P.units = reinterpret_cast<const int4*>(compact ? m->tau_units_split[k] : m->tau_units[k]);
      P.n_list = phase == 0 ? c.n : (compact ? m->tau_n_units_split[k] : m->tau_n_units[k]);
      if (phase == 1) {
        m->tau_last_units[k] = P.n_list;
        m->tau_last_shared[k] = compact ? 0 : m->tau_n_shared[k];
      }
      if (P.n_list == 0) continue;
      const size_t smem = tau_smem_for(c.S, ns, fp32, compact);
      const int grid = grid_for(P.n_list, 16);
#define DG_TAU_CASE(AFF, NSV, AXV)                                                             \
  if (phase == 0) {                                                                             \
    if ((err = allow_smem(tau_prologue_kernel<T, AFF, NSV, AXV>, smem))) return err;            \
    tau_prologue_kernel<T, AFF, NSV, AXV><<<grid, kVolThreads, smem, m->stream>>>(P);           \
  } else {                                                                                      \
    if ((err = allow_smem(tau_kernel<T, AFF, NSV, AXV>, smem))) return err;                     \
    tau_kernel<T, AFF, NSV, AXV><<<grid, kVolThreads, smem, m->stream>>>(P);                    \
  }
#define DG_TAU_EULER_T(AFF, AXV, TH)                                                            \
  if (phase == 0) {                                                                             \
    if ((err = allow_smem(tau_euler_prologue_kernel<T, AFF, AXV, TH>, smem))) return err;       \
    tau_euler_prologue_kernel<T, AFF, AXV, TH><<<grid, TH, smem, m->stream>>>(P);              \
  } else {                                                                                      \
    if ((err = allow_smem(tau_euler_kernel<T, AFF, AXV, TH>, smem))) return err;                \
    tau_euler_kernel<T, AFF, AXV, TH><<<grid, TH, smem, m->stream>>>(P);                       \
  }
      // the Euler sweep's CTA grows when shared memory admits fewer CTAs per SM,
      // so that every class keeps ~32 warps per SM (FP32; FP64 as registers allow)
      const int threads = tau_euler_threads(smem + tau_static_bytes(fp32), fp32);
      constexpr int kTauMaxThreads = sizeof(T) == 4 ? 1024 : 512;
#define DG_TAU_EULER(AFF, AXV)                                                                  \
  if (threads >= 1024) { DG_TAU_EULER_T(AFF, AXV, kTauMaxThreads) }                             \
  else if (threads >= 512) { DG_TAU_EULER_T(AFF, AXV, 512) }                                    \
  else { DG_TAU_EULER_T(AFF, AXV, 256) }
      if (m->axis && !ns) { DG_TAU_EULER(true, true) }
      else if (m->affine && !ns) { DG_TAU_EULER(true, false) }
      else if (!ns) { DG_TAU_EULER(false, false) }
      else if (m->affine) { DG_TAU_CASE(true, true, false) }
      else { DG_TAU_CASE(false, true, false) }
#undef DG_TAU_CASE
#undef DG_TAU_EULER
#undef DG_TAU_EULER_T
      if ((err = cudaGetLastError())) return err;
    }
  }
  return cudaSuccess;
}

cudaError_t tau_isolated(dg_mesh_impl* m, const double* q, const double* r_p, const int32_t* d_sweep, int n_sweep,
                         bool fp32, bool accumulate, void* map_new, void* map_trad) {
  auto fill = [&](auto& P) {
    P.m = view(m);
    P.n_elem = m->n_elem;
    P.q = q;
    P.rp = r_p;
    P.sweep = d_sweep;
    P.n_sweep = n_sweep;
    P.accumulate = accumulate;
    P.gamma = m->phys.gamma;
    P.mu = m->phys.mu;
    P.Pr = m->phys.Pr;
    P.Rgas = m->phys.Rgas;
    P.kappa_R = m->phys.kappa_R;
    P.gamma64 = m->phys.gamma;
    P.err = m->d_err;
    P.bank_off = m->d_taugeo_off;
  };
  if (fp32) {
    TauParams<float> P;
    fill(P);
    P.basis = m->basis32;
    P.metric = m->affine ? m->d_metric32 : m->d_taugeo32;
    P.map_new = static_cast<float*>(map_new);
    P.map_trad = static_cast<float*>(map_trad);
    P.rp_scratch = m->d_rp32;
    return tau_launch(m, P, true);
  }
  TauParams<double> P;
  fill(P);
  P.basis = m->basis64;
  P.metric = m->affine ? m->d_metric : m->d_taugeo;
  P.map_new = static_cast<double*>(map_new);
  P.map_trad = static_cast<double*>(map_trad);
  P.rp_scratch = m->d_rp;
  return tau_launch(m, P, false);
}

cudaError_t tau_combine(dg_mesh_impl* m, dg_mesh_impl* c, const double* r_p, const double* r_c, int s, int n_sweep,
                        const int32_t* h_sweep, bool fp32, bool accumulate, void* map_new, void* map_trad) {
  int S = 1;
  for (int e = 0; e < m->n_elem; ++e) {
    int n = (m->h_ord[3 * e] + 1) * (m->h_ord[3 * e + 1] + 1) * (m->h_ord[3 * e + 2] + 1);
    if (n > S) S = n;
  }
  size_t smem = sizeof(double) * 15 * S;
  int grid = grid_for(m->n_elem, 4);
  int N1 = h_sweep[3 * s], N2 = h_sweep[3 * s + 1], N3 = h_sweep[3 * s + 2];
  cudaError_t err;
  Prof pr(m, DG_KERNEL_TAU_COMBINE);
#define DG_COMB(MT, AFF)                                                                                     \
  if ((err = allow_smem(tau_combine_kernel<MT, AFF>, smem))) return err;                                      \
  tau_combine_kernel<MT, AFF><<<grid, kTauThreads, smem, m->stream>>>(                                        \
      view(m), view(c), r_p, r_c, m->basis64, N1, N2, N3, s, n_sweep, S, accumulate, static_cast<MT*>(map_new), \
      static_cast<MT*>(map_trad), m->n_elem);
  if (fp32 && m->affine) { DG_COMB(float, true) }
  else if (fp32) { DG_COMB(float, false) }
  else if (m->affine) { DG_COMB(double, true) }
  else { DG_COMB(double, false) }
#undef DG_COMB
  return cudaGetLastError();
}

cudaError_t project_orders(dg_mesh_impl* m, const int32_t* d_new_orders, const int64_t* d_new_off,
                           const double* q_old, double* q_new, int mode) {
  const int S = (DG_MAX_ORDER + 1) * (DG_MAX_ORDER + 1) * (DG_MAX_ORDER + 1);
  size_t smem = sizeof(double) * 10 * S;
  int grid = grid_for(m->n_elem, 4);
  cudaError_t err = allow_smem(project_kernel, smem);
  if (err) return err;
  Prof pr(m, DG_KERNEL_PROJECT);
  project_kernel<<<grid, kTauThreads, smem, m->stream>>>(m->d_ord, m->d_off, d_new_orders, d_new_off, m->basis64, q_old,
                                                          q_new, m->n_elem, S, mode);
  return cudaGetLastError();
}

}  // namespace dgk

// ---------------------------------------------------------------------------
// dg_residual_noalloc: the Euler residual with its face-flux scratch in a
// fixed device array instead of the mesh's buffer, for callers that may not
// allocate device memory.
// ---------------------------------------------------------------------------

// 4 Mi doubles (32 MiB): the face buffer of up to 838,860 element-face nodes
// (5 doubles each).  Every GPU that loads the library holds it until exit.
static_assert(DG_NOALLOC_SURF_DOUBLES == (4u << 20), "fixed face-buffer size");
static __device__ __align__(256) double g_noalloc_surf[DG_NOALLOC_SURF_DOUBLES];

// Device address of g_noalloc_surf on device dev.  In host code the array's
// name is only a host-side stand-in, so the address is looked up with that
// device current (the caller's current device).  Outside stream capture every
// call looks it up again, so an address never outlives the context it came
// from (a cudaDeviceReset in the caller makes a new one); while the stream is
// being captured the address of the last lookup on this device is used.  The
// per-device entries are atomics: two host threads may make their first call
// at the same time.
static std::atomic<double*> g_noalloc_addr[64];

static double* noalloc_surf_address(int dev, cudaStream_t stream, cudaError_t* err) {
  *err = cudaSuccess;
  if (dev < 0 || dev >= 64) {
    *err = cudaErrorInvalidDevice;
    return nullptr;
  }
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  if ((*err = cudaStreamIsCapturing(stream, &cs)) != cudaSuccess) return nullptr;
  if (cs != cudaStreamCaptureStatusNone) {
    double* p = g_noalloc_addr[dev].load(std::memory_order_acquire);
    if (!p) *err = cudaErrorStreamCaptureUnsupported;   // no lookup made on this device before the capture
    return p;
  }
  void* p = nullptr;
  if ((*err = cudaGetSymbolAddress(&p, g_noalloc_surf)) != cudaSuccess) return nullptr;
  g_noalloc_addr[dev].store(static_cast<double*>(p), std::memory_order_release);
  return static_cast<double*>(p);
}

extern "C" dg_status dg_residual_noalloc(dg_mesh* mesh, const double* q, double* r) {
  if (!mesh || !q || !r || q == r) return DG_ERR_ARG;
  if (mesh->phys.eqs != DG_EULER || mesh->faces_unsupported) return DG_ERR_UNSUPPORTED;
  const size_t need = 5 * (size_t)mesh->h_soff[mesh->n_elem];
  if (need > DG_NOALLOC_SURF_DOUBLES) return DG_ERR_UNSUPPORTED;   // mesh too large for the fixed buffer
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return DG_ERR_CUDA;
  if (dev != mesh->device) return DG_ERR_ARG;                      // the mesh's device must be current
  cudaError_t err;
  double* surf = noalloc_surf_address(dev, mesh->stream, &err);
  if (!surf) return DG_ERR_CUDA;
  // face pass: every element-face node of the buffer is written (interior
  // faces for both sides, boundary faces for theirs) before the volume pass
  // reads it, so nothing needs clearing between calls
  if (launch_all_faces(mesh, q, nullptr, surf) != cudaSuccess) return DG_ERR_CUDA;
  VolParams V = dgk_vol_params_for(mesh, q, surf, r);
  size_t vsmem = 0;
  int vgrid = 0;
  if (dispatch_volume(mesh, V, vsmem, vgrid) != cudaSuccess) return DG_ERR_CUDA;
  mesh->launches += (int64_t)mesh->vol_classes.size();   // the face launches count themselves
  return cudaGetLastError() == cudaSuccess ? DG_OK : DG_ERR_CUDA;
}

// ---------------------------------------------------------------------------
// Static p-adaptation (Sec. 2.4, approach 2): order selection from a total
// truncation-error map and the degree-jump conditions of Sec. 3.1.
// ---------------------------------------------------------------------------
namespace {

// Per element: the sweep entry with 0 <= map < tau_max and n_min <= N_i <=
// n_max of fewest degrees of freedom prod_i (N_i+1), the first in sweep
// order on ties; n_max in every direction when none qualifies.
template <typename T>
__global__ void select_kernel(const T* map, const int32_t* sweep, int n_sweep, int n_elem, double tau_max, int n_min,
                              int n_max, const int32_t* prev, int max_decrease, int32_t* out) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_elem) return;
  long long best = -1;
  int bs = -1;
  const T* row = map + (int64_t)e * n_sweep;
  for (int s = 0; s < n_sweep; ++s) {
    const double v = (double)row[s];
    const int N0 = sweep[3 * s], N1 = sweep[3 * s + 1], N2 = sweep[3 * s + 2];
    if (!(v >= 0.0 && v < tau_max)) continue;
    if (N0 < n_min || N1 < n_min || N2 < n_min || N0 > n_max || N1 > n_max || N2 > n_max) continue;
    const long long nd = (long long)(N0 + 1) * (N1 + 1) * (N2 + 1);
    if (best < 0 || nd < best) {
      best = nd;
      bs = s;
    }
  }
  for (int d = 0; d < 3; ++d) {
    int o = bs >= 0 ? sweep[3 * bs + d] : n_max;
    if (max_decrease >= 0) {   // dynamic adaptation: fall by at most max_decrease below the current order
      int lo = prev[3 * e + d] - max_decrease;
      lo = lo > n_max ? n_max : lo;
      o = o < lo ? lo : o;
    }
    out[3 * e + d] = o;
  }
}

// One Jacobi sweep of the jump condition: rule 1 (Eq. N23) N_i^e >=
// floor(2 N_i^j / 3), rule 2 (Eq. N_1) N_i^e >= N_i^j - 1 over the face
// neighbours j; sets *changed when an order rose.
__global__ void jump_kernel(const int32_t* cur, int32_t* nxt, const int32_t* nbr, int n_elem, int rule,
                            int* changed) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= n_elem) return;
  for (int d = 0; d < 3; ++d) {
    int need = cur[3 * e + d];
    for (int f = 0; f < 6; ++f) {
      const int j = nbr[6 * e + f];
      if (j < 0) continue;
      const int nj = cur[3 * j + d];
      const int lim = rule == 1 ? (2 * nj) / 3 : nj - 1;
      need = lim > need ? lim : need;
    }
    if (need != cur[3 * e + d]) *changed = 1;
    nxt[3 * e + d] = need;
  }
}

}  // namespace

extern "C" dg_status dg_select_orders(dg_mesh* m, const void* map, int32_t map_fp32, const int32_t* sweep,
                                      int32_t n_sweep, double tau_max, int32_t n_min, int32_t n_max,
                                      int32_t jump_rule, int32_t max_decrease, int32_t* orders_out) {
  if (!m || !map || !sweep || n_sweep <= 0 || !orders_out || !(tau_max > 0.0)) return DG_ERR_ARG;
  if (n_min < 1 || n_max > DG_MAX_ORDER || n_min > n_max || jump_rule < 0 || jump_rule > 2) return DG_ERR_ARG;
  for (int s = 0; s < 3 * n_sweep; ++s)
    if (sweep[s] < 1 || sweep[s] > DG_MAX_ORDER) return DG_ERR_ARG;
  const int ne = m->n_elem;
  int32_t *d_sw = nullptr, *d_a = nullptr, *d_b = nullptr;
  int* d_flag = nullptr;
  dg_status st = DG_OK;
  auto fail = [&](cudaError_t e) { st = e == cudaErrorMemoryAllocation ? DG_ERR_NOMEM : DG_ERR_CUDA; };
  cudaError_t e;
  if ((e = cudaMalloc(&d_sw, sizeof(int32_t) * 3 * n_sweep)) || (e = cudaMalloc(&d_a, sizeof(int32_t) * 3 * ne)) ||
      (e = cudaMalloc(&d_b, sizeof(int32_t) * 3 * ne)) || (e = cudaMalloc(&d_flag, sizeof(int)))) {
    fail(e);
  } else if ((e = cudaMemcpyAsync(d_sw, sweep, sizeof(int32_t) * 3 * n_sweep, cudaMemcpyHostToDevice, m->stream))) {
    fail(e);
  } else {
    const int grid = (ne + 127) / 128;
    dg_prof_begin(m, DG_KERNEL_SELECT, 1);
    if (map_fp32)
      select_kernel<float><<<grid, 128, 0, m->stream>>>(static_cast<const float*>(map), d_sw, n_sweep, ne, tau_max,
                                                         n_min, n_max, m->d_ord, max_decrease, d_a);
    else
      select_kernel<double><<<grid, 128, 0, m->stream>>>(static_cast<const double*>(map), d_sw, n_sweep, ne,
                                                          tau_max, n_min, n_max, m->d_ord, max_decrease, d_a);
    dg_prof_end(m, DG_KERNEL_SELECT);
    if ((e = cudaGetLastError())) fail(e);
    // jump condition: Jacobi sweeps to the least fixed point (orders only
    // rise, bounded by n_max, so at most n_max * n_elem sweeps; in practice
    // a few)
    for (int it = 0; st == DG_OK && jump_rule && it <= DG_MAX_ORDER * ne + 1; ++it) {
      int flag = 0;
      if ((e = cudaMemsetAsync(d_flag, 0, sizeof(int), m->stream))) { fail(e); break; }
      dg_prof_begin(m, DG_KERNEL_SELECT, 1);
      jump_kernel<<<grid, 128, 0, m->stream>>>(d_a, d_b, m->d_nbr, ne, jump_rule, d_flag);
      dg_prof_end(m, DG_KERNEL_SELECT);
      if ((e = cudaGetLastError())) { fail(e); break; }
      if ((e = cudaMemcpyAsync(&flag, d_flag, sizeof(int), cudaMemcpyDeviceToHost, m->stream))) { fail(e); break; }
      if ((e = cudaStreamSynchronize(m->stream))) { fail(e); break; }
      std::swap(d_a, d_b);
      if (!flag) break;
    }
    if (st == DG_OK) {
      if ((e = cudaMemcpyAsync(orders_out, d_a, sizeof(int32_t) * 3 * ne, cudaMemcpyDeviceToHost, m->stream)))
        fail(e);
      else if ((e = cudaStreamSynchronize(m->stream)))
        fail(e);
    }
  }
  cudaFree(d_sw);
  cudaFree(d_a);
  cudaFree(d_b);
  cudaFree(d_flag);
  return st;
}

// ---------------------------------------------------------------------------
// Adjoint (vector-Jacobian product) of the residual, Euler on straight-sided
// elements.  R = A Phi(q): Phi the pointwise fluxes (contravariant volume
// flux at the nodes, Roe at the face and mortar nodes), A linear (GL
// derivative, surface lift, mortar interpolation and L2 projection, -1/J).
// J^T v = (dPhi/dq)^T A^T v: the kernels apply the transposes of the linear
// steps and take (dPhi/dq)^T from Jacobian columns computed by running the
// same flux functions on Dual numbers, one input component seeded at a time.
// ---------------------------------------------------------------------------
namespace {

template <typename S>
__device__ __forceinline__ void euler_flux3(double gm1, const S q[5], S f[3][5]) {
  const S ir = 1.0 / q[0];
  const S u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  const S p = gm1 * (q[4] - 0.5 * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
  for (int d = 0; d < 3; ++d) {
    f[d][0] = q[1 + d];
    f[d][1] = q[1] * u[d];
    f[d][2] = q[2] * u[d];
    f[d][3] = q[3] * u[d];
    f[d][1 + d] += p;
    f[d][4] = u[d] * (q[4] + p);
  }
}

template <bool AXIS>
__device__ __forceinline__ void roe_face_d(double gamma, int dir, const Dual qL[5], const Dual qR[5],
                                           const double n[3], Dual f[5]) {
  if (AXIS) {
    if (dir == 0) roe_t<0, Dual>(gamma, qL, qR, n, f, 0.5);
    else if (dir == 1) roe_t<1, Dual>(gamma, qL, qR, n, f, 0.5);
    else roe_t<2, Dual>(gamma, qL, qR, n, f, 0.5);
  } else {
    roe_t<-1, Dual>(gamma, qL, qR, n, f, 0.5);
  }
}

// The Roe flux's vector-Jacobian product by a reverse (adjoint) sweep: the
// forward quantities of roe_t, then their cotangents in reverse order, each
// step the transpose of one forward line.  gL = (dF/dqL)^T lf, gR likewise;
// the same derivative the Dual evaluations give (|x| at x = 0 takes the
// derivative of +x, as absval does), at a few times the cost of one flux.
template <int AX>
__device__ void roe_vjp_rev(double gamma, const double qL[5], const double qR[5], const double n[3],
                            const double lf[5], double gL[5], double gR[5]) {
  const double gm1 = gamma - 1.0;
  // forward
  const double rsL = rsqrt(qL[0]), rsR = rsqrt(qR[0]);
  const double sL = qL[0] * rsL, sR = qR[0] * rsR;
  const double irL = rsL * rsL, irR = rsR * rsR;
  double uL[3], uR[3], nc[3];
  for (int c = 0; c < 3; ++c) {
    uL[c] = qL[1 + c] * irL;
    uR[c] = qR[1 + c] * irR;
    nc[c] = ncomp<AX>(n, c);
  }
  const double pL = gm1 * (qL[4] - 0.5 * (qL[1] * uL[0] + qL[2] * uL[1] + qL[3] * uL[2]));
  const double pR = gm1 * (qR[4] - 0.5 * (qR[1] * uR[0] + qR[2] * uR[1] + qR[3] * uR[2]));
  const double HL = (qL[4] + pL) * irL, HR = (qR[4] + pR) * irR;
  const double is = 1.0 / (sL + sR);
  double ut[3];
  for (int c = 0; c < 3; ++c) ut[c] = (sL * uL[c] + sR * uR[c]) * is;
  const double Ht = (sL * HL + sR * HR) * is;
  const double rt = sL * sR;
  const double q2 = ut[0] * ut[0] + ut[1] * ut[1] + ut[2] * ut[2];
  const double c2 = gm1 * (Ht - 0.5 * q2);
  const double rc = rsqrt(c2);
  const double ct = c2 * rc, ic2 = rc * rc;
  const double unL = uL[0] * nc[0] + uL[1] * nc[1] + uL[2] * nc[2];
  const double unR = uR[0] * nc[0] + uR[1] * nc[1] + uR[2] * nc[2];
  const double utn = ut[0] * nc[0] + ut[1] * nc[1] + ut[2] * nc[2];
  const double dun = unR - unL, dp = pR - pL;
  const double rcd = rt * ct * dun;
  const double a1 = 0.5 * (dp - rcd) * ic2, a5 = 0.5 * (dp + rcd) * ic2;
  const double a2 = (qR[0] - qL[0]) - dp * ic2;
  const double s1 = (utn - ct) < 0.0 ? -1.0 : 1.0, s5 = (utn + ct) < 0.0 ? -1.0 : 1.0, s2 = utn < 0.0 ? -1.0 : 1.0;
  const double l1 = s1 * (utn - ct), l5 = s5 * (utn + ct), l2 = s2 * utn;
  const double l1a1 = l1 * a1, l5a5 = l5 * a5;
  double dut[3], utdut = 0.0;
  for (int c = 0; c < 3; ++c) {
    dut[c] = (uR[c] - uL[c]) - dun * nc[c];
    utdut += ut[c] * dut[c];
  }
  const double mL = qL[0] * unL, mR = qR[0] * unR;
  // reverse
  double mL_b = 0.5 * lf[0], mR_b = 0.5 * lf[0];
  double l1a1_b = -0.5 * lf[0], l5a5_b = -0.5 * lf[0];
  double l2_b = -0.5 * lf[0] * a2, a2_b = -0.5 * lf[0] * l2;
  double uL_b[3] = {0, 0, 0}, uR_b[3] = {0, 0, 0}, ut_b[3] = {0, 0, 0}, dut_b[3] = {0, 0, 0};
  double pL_b = 0.0, pR_b = 0.0, ct_b = 0.0, rt_b = 0.0, Ht_b = 0.0, utn_b = 0.0, q2_b = 0.0, utdut_b = 0.0;
  double unL_b = 0.0, unR_b = 0.0, qL4_b = 0.0, qR4_b = 0.0;
  {  // f4 = 0.5 (physE - dissE)
    const double pe = 0.5 * lf[4], de = -0.5 * lf[4];
    unL_b += pe * (qL[4] + pL);
    qL4_b += pe * unL;
    pL_b += pe * unL;
    unR_b += pe * (qR[4] + pR);
    qR4_b += pe * unR;
    pR_b += pe * unR;
    l1a1_b += de * (Ht - utn * ct);
    l5a5_b += de * (Ht + utn * ct);
    Ht_b += de * (l1a1 + l5a5);
    utn_b += de * (l5a5 - l1a1) * ct;
    ct_b += de * (l5a5 - l1a1) * utn;
    l2_b += de * (a2 * 0.5 * q2 + rt * utdut);
    a2_b += de * l2 * 0.5 * q2;
    q2_b += de * l2 * 0.5 * a2;
    rt_b += de * l2 * utdut;
    utdut_b += de * l2 * rt;
  }
  for (int c = 0; c < 3; ++c) {  // f[1+c] = 0.5 (phys_c - diss_c)
    const double ph = 0.5 * lf[1 + c], di = -0.5 * lf[1 + c];
    mL_b += ph * uL[c];
    uL_b[c] += ph * mL;
    mR_b += ph * uR[c];
    uR_b[c] += ph * mR;
    pL_b += ph * nc[c];
    pR_b += ph * nc[c];
    l1a1_b += di * (ut[c] - ct * nc[c]);
    l5a5_b += di * (ut[c] + ct * nc[c]);
    ut_b[c] += di * (l1a1 + l5a5 + l2 * a2);
    l2_b += di * (a2 * ut[c] + rt * dut[c]);
    a2_b += di * l2 * ut[c];
    rt_b += di * l2 * dut[c];
    dut_b[c] += di * l2 * rt;
    ct_b += di * (l5a5 - l1a1) * nc[c];
  }
  double qL0_b = mL_b * unL, qR0_b = mR_b * unR;
  unL_b += mL_b * qL[0];
  unR_b += mR_b * qR[0];
  double dun_b = 0.0;
  for (int c = 0; c < 3; ++c) {
    ut_b[c] += utdut_b * dut[c];
    dut_b[c] += utdut_b * ut[c];
    uR_b[c] += dut_b[c];
    uL_b[c] -= dut_b[c];
    dun_b -= dut_b[c] * nc[c];
  }
  const double l1_b = l1a1_b * a1, l5_b = l5a5_b * a5;
  double a1_b = l1a1_b * l1, a5_b = l5a5_b * l5;
  utn_b += l1_b * s1 + l5_b * s5 + l2_b * s2;
  ct_b += -l1_b * s1 + l5_b * s5;
  double dp_b = -a2_b * ic2, ic2_b = -a2_b * dp;
  qR0_b += a2_b;
  qL0_b -= a2_b;
  dp_b += 0.5 * ic2 * (a1_b + a5_b);
  double rcd_b = 0.5 * ic2 * (a5_b - a1_b);
  ic2_b += 0.5 * (a1_b * (dp - rcd) + a5_b * (dp + rcd));
  rt_b += rcd_b * ct * dun;
  ct_b += rcd_b * rt * dun;
  dun_b += rcd_b * rt * ct;
  unR_b += dun_b;
  unL_b -= dun_b;
  pR_b += dp_b;
  pL_b -= dp_b;
  for (int c = 0; c < 3; ++c) {
    ut_b[c] += utn_b * nc[c];
    uL_b[c] += unL_b * nc[c];
    uR_b[c] += unR_b * nc[c];
  }
  double rc_b = ct_b * c2 + ic2_b * 2.0 * rc;
  double c2_b = ct_b * rc - 0.5 * rc_b * rc * rc * rc;
  Ht_b += c2_b * gm1;
  q2_b -= c2_b * 0.5 * gm1;
  for (int c = 0; c < 3; ++c) ut_b[c] += q2_b * 2.0 * ut[c];
  double sL_b = rt_b * sR, sR_b = rt_b * sL;
  double is_b = Ht_b * (sL * HL + sR * HR);
  sL_b += Ht_b * HL * is;
  sR_b += Ht_b * HR * is;
  const double HL_b = Ht_b * sL * is, HR_b = Ht_b * sR * is;
  for (int c = 0; c < 3; ++c) {
    sL_b += ut_b[c] * uL[c] * is;
    uL_b[c] += ut_b[c] * sL * is;
    sR_b += ut_b[c] * uR[c] * is;
    uR_b[c] += ut_b[c] * sR * is;
    is_b += ut_b[c] * (sL * uL[c] + sR * uR[c]);
  }
  const double ss_b = -is_b * is * is;
  sL_b += ss_b;
  sR_b += ss_b;
  // HL = (qL4 + pL) irL
  qL4_b += HL_b * irL;
  pL_b += HL_b * irL;
  double irL_b = HL_b * (qL[4] + pL);
  qR4_b += HR_b * irR;
  pR_b += HR_b * irR;
  double irR_b = HR_b * (qR[4] + pR);
  // p = gm1 (q4 - 0.5 sum_c q[1+c] u[c])
  double qLm_b[3], qRm_b[3];
  qL4_b += pL_b * gm1;
  qR4_b += pR_b * gm1;
  for (int c = 0; c < 3; ++c) {
    qLm_b[c] = -pL_b * gm1 * 0.5 * uL[c];
    uL_b[c] -= pL_b * gm1 * 0.5 * qL[1 + c];
    qRm_b[c] = -pR_b * gm1 * 0.5 * uR[c];
    uR_b[c] -= pR_b * gm1 * 0.5 * qR[1 + c];
    // u = q[1+c] ir
    qLm_b[c] += uL_b[c] * irL;
    irL_b += uL_b[c] * qL[1 + c];
    qRm_b[c] += uR_b[c] * irR;
    irR_b += uR_b[c] * qR[1 + c];
  }
  // ir = rs^2, s = q0 rs, rs = q0^(-1/2)
  double rsL_b = irL_b * 2.0 * rsL + sL_b * qL[0], rsR_b = irR_b * 2.0 * rsR + sR_b * qR[0];
  qL0_b += sL_b * rsL - 0.5 * rsL_b * rsL * rsL * rsL;
  qR0_b += sR_b * rsR - 0.5 * rsR_b * rsR * rsR * rsR;
  gL[0] = qL0_b;
  gR[0] = qR0_b;
  for (int c = 0; c < 3; ++c) {
    gL[1 + c] = qLm_b[c];
    gR[1 + c] = qRm_b[c];
  }
  gL[4] = qL4_b;
  gR[4] = qR4_b;
}

// gL[k] = sum_v dF_v/dqL_k lf_v, gR likewise: the Roe flux's Jacobian
// transposes applied to lf (the reverse sweep above)
template <bool AXIS>
__device__ void roe_vjp(double gamma, int dir, const double qL[5], const double qR[5], const double n[3],
                        const double lf[5], double gL[5], double gR[5]) {
  if (AXIS) {
    if (dir == 0) roe_vjp_rev<0>(gamma, qL, qR, n, lf, gL, gR);
    else if (dir == 1) roe_vjp_rev<1>(gamma, qL, qR, n, lf, gL, gR);
    else roe_vjp_rev<2>(gamma, qL, qR, n, lf, gL, gR);
  } else {
    roe_vjp_rev<-1>(gamma, qL, qR, n, lf, gL, gR);
  }
}

// 1 / w_0 = 1 / w_N of the order-N GL rule
__device__ __forceinline__ double inv_wend(int N) { return 0.5 * N * (N + 1); }

// Mortar batches, reversed.  Per batch: the traces and the face cotangents
// lf_side = s_side (1/w_N) (-v/J) at each side's face nodes (s = +1 behind
// the face, -1 ahead: the sign of the lift), the forward interpolation up
// to the mortar (the Roe linearisation point), the transposes of the two
// projection passes onto the mortar grid (both sides summed), the Roe
// vector-Jacobian product at the mortar nodes, and the transposes of the two
// interpolation passes back onto each side's face grid, into sadj.
// shared memory (doubles) of an adjoint mortar batch
__host__ __device__ inline size_t mortar_adj_smem_doubles(int count, int la, int lb, int ra, int rb) {
  const int Ma = la > ra ? la : ra, Mb = lb > rb ? lb : rb;
  const int uL = (Ma * lb > la * Mb ? Ma * lb : la * Mb), uR = (Ma * rb > ra * Mb ? Ma * rb : ra * Mb);
  return (size_t)count * (5 * (2 * la * lb + 2 * ra * rb + uL + uR + 3 * Ma * Mb) + 4);
}

template <bool AXIS>
__global__ void __launch_bounds__(kVolThreads) adj_mortar_kernel(MortarParams P, const double* __restrict__ vin,
                                                                 double* __restrict__ sadj) {
  extern __shared__ double smem[];
  const MeshView& m = P.m;
  const double gamma = m.ph.gamma;
  for (int it = blockIdx.x; it < P.n_batches; it += gridDim.x) {
    const MortarBatch B = P.batches[it];
    if (bad_batch(P, B, mortar_adj_smem_doubles(B.count, B.la, B.lb, B.ra, B.rb))) continue;
    const int la = B.la, lb = B.lb, ra = B.ra, rb = B.rb, cnt = B.count;
    const int Ma = la > ra ? la : ra, Mb = lb > rb ? lb : rb;
    const int nfl = la * lb, nfr = ra * rb, nm = Ma * Mb;
    const bool upLa = la != Ma, upLb = lb != Mb, upRa = ra != Ma, upRb = rb != Mb;
    const int uL = (Ma * lb > la * Mb ? Ma * lb : la * Mb), uR = (Ma * rb > ra * Mb ? Ma * rb : ra * Mb);
    double* TL = smem;
    double* TR = TL + cnt * 5 * nfl;
    double* UL = TR + cnt * 5 * nfr;
    double* UR = UL + cnt * 5 * uL;
    double* QL = UR + cnt * 5 * uR;
    double* QR = QL + cnt * 5 * nm;
    double* AL = QR + cnt * 5 * nm;   // face cotangents on each side's grid
    double* AR = AL + cnt * 5 * nfl;
    double* LM = AR + cnt * 5 * nfr;  // flux cotangent at the mortar nodes
    double* NR = LM + cnt * 5 * nm;
    // 1. traces, face cotangents, normals
    for (int t = threadIdx.x; t < cnt * (nfl + nfr); t += blockDim.x) {
      const bool isL = t < cnt * nfl;
      const int tt = isL ? t : t - cnt * nfl;
      const int nf = isL ? nfl : nfr, na = isL ? la : ra;
      const int f = tt / nf, p = tt - f * nf;
      const int* fr = P.faces + 3 * (B.first + f);
      const int e = isL ? fr[0] : fr[1], dir = fr[2];
      int n1, n2, n3;
      orders_of(m, e, n1, n2, n3);
      const int n = n1 * n2 * n3;
      const int vi = face_vidx(n1, n2, n3, isL ? 2 * dir + 1 : 2 * dir, p % na, p / na);
      const int64_t o = m.off[e];
      const int Nd = (dir == 0 ? n1 : dir == 1 ? n2 : n3) - 1;
      const double c = (isL ? -1.0 : 1.0) * inv_wend(Nd) * metric<true>(m.metric, e, 0, 0, 0, 10);
      double* T = (isL ? TL + f * 5 * nfl : TR + f * 5 * nfr) + p;
      double* A = (isL ? AL + f * 5 * nfl : AR + f * 5 * nfr) + p;
      for (int v = 0; v < 5; ++v) {
        T[v * nf] = P.q[5 * o + v * n + vi];
        A[v * nf] = c * vin[5 * o + v * n + vi];
      }
    }
    for (int f = threadIdx.x; f < cnt; f += blockDim.x) {
      const int* fr = P.faces + 3 * (B.first + f);
      double ja[3], nrm[3];
      for (int c = 0; c < 3; ++c) ja[c] = metric<true>(m.metric, fr[0], 0, 0, 0, 3 * fr[2] + c);
      const double area = unit_normal(ja, nrm);
      NR[4 * f + 0] = nrm[0];
      NR[4 * f + 1] = nrm[1];
      NR[4 * f + 2] = nrm[2];
      NR[4 * f + 3] = area;
    }
    __syncthreads();
    // 2-3. interpolation up to the mortar, as in the forward kernel
    const double* IaL = P.basis + c_boff.I[la - 1][Ma - 1];
    const double* IaR = P.basis + c_boff.I[ra - 1][Ma - 1];
    const double* IbL = P.basis + c_boff.I[lb - 1][Mb - 1];
    const double* IbR = P.basis + c_boff.I[rb - 1][Mb - 1];
    {
      const int nL = upLa ? cnt * Ma * lb : 0, nR = upRa ? cnt * Ma * rb : 0;
      for (int t = threadIdx.x; t < nL + nR; t += blockDim.x) {
        const bool isL = t < nL;
        const int tt = isL ? t : t - nL;
        const int nb = isL ? lb : rb, na = isL ? la : ra, per = Ma * nb;
        const int f = tt / per, x = tt - f * per, m0 = x % Ma, b = x / Ma;
        const double* src = isL ? TL + f * 5 * nfl : TR + f * 5 * nfr;
        const double* Ia = isL ? IaL : IaR;
        double* dst = (isL ? UL + f * 5 * uL : UR + f * 5 * uR) + x;
        const int nsrc = na * nb;
        double acc[5] = {0, 0, 0, 0, 0};
        for (int a = 0; a < na; ++a) {
          const double w = __ldg(Ia + m0 * na + a);
          for (int v = 0; v < 5; ++v) acc[v] += w * src[v * nsrc + a + na * b];
        }
        for (int v = 0; v < 5; ++v) dst[v * per] = acc[v];
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * cnt * nm; t += blockDim.x) {
      const bool isL = t < cnt * nm;
      const int tt = isL ? t : t - cnt * nm;
      const int f = tt / nm, x = tt - f * nm, m0 = x % Ma, m1 = x / Ma;
      const bool upa = isL ? upLa : upRa, upb = isL ? upLb : upRb;
      const int nb = isL ? lb : rb;
      const double* src = upa ? (isL ? UL + f * 5 * uL : UR + f * 5 * uR) : (isL ? TL + f * 5 * nfl : TR + f * 5 * nfr);
      const int nsrc = Ma * nb;
      double* dst = (isL ? QL : QR) + f * 5 * nm + x;
      if (upb) {
        const double* Ib = isL ? IbL : IbR;
        double acc[5] = {0, 0, 0, 0, 0};
        for (int b = 0; b < nb; ++b) {
          const double w = __ldg(Ib + m1 * nb + b);
          for (int v = 0; v < 5; ++v) acc[v] += w * src[v * nsrc + m0 + Ma * b];
        }
        for (int v = 0; v < 5; ++v) dst[v * nm] = acc[v];
      } else {
        for (int v = 0; v < 5; ++v) dst[v * nm] = src[v * nsrc + m0 + Ma * m1];
      }
    }
    __syncthreads();
    // 4a. transpose of the xi_b projection pass: X(a, m1) = sum_b Pb(b, m1) A(a, b), into U
    const double* PaL = P.basis + c_boff.P[Ma - 1][la - 1];
    const double* PaR = P.basis + c_boff.P[Ma - 1][ra - 1];
    const double* PbL = P.basis + c_boff.P[Mb - 1][lb - 1];
    const double* PbR = P.basis + c_boff.P[Mb - 1][rb - 1];
    {
      const int nL = upLb ? cnt * la * Mb : 0, nR = upRb ? cnt * ra * Mb : 0;
      for (int t = threadIdx.x; t < nL + nR; t += blockDim.x) {
        const bool isL = t < nL;
        const int tt = isL ? t : t - nL;
        const int na = isL ? la : ra, nb = isL ? lb : rb, per = na * Mb;
        const int f = tt / per, x = tt - f * per, a = x % na, m1 = x / na;
        const double* Pb = isL ? PbL : PbR;
        const double* src = isL ? AL + f * 5 * nfl : AR + f * 5 * nfr;
        double* dst = (isL ? UL + f * 5 * uL : UR + f * 5 * uR) + x;
        const int nsrc = na * nb;
        double acc[5] = {0, 0, 0, 0, 0};
        for (int b = 0; b < nb; ++b) {
          const double w = __ldg(Pb + b * Mb + m1);
          for (int v = 0; v < 5; ++v) acc[v] += w * src[v * nsrc + a + na * b];
        }
        for (int v = 0; v < 5; ++v) dst[v * per] = acc[v];
      }
    }
    __syncthreads();
    // 4b. transpose of the xi_a projection pass, both sides summed onto the mortar grid
    for (int t = threadIdx.x; t < cnt * nm; t += blockDim.x) {
      const int f = t / nm, x = t - f * nm, m0 = x % Ma, m1 = x / Ma;
      double acc[5] = {0, 0, 0, 0, 0};
      for (int side = 0; side < 2; ++side) {
        const bool isL = side == 0;
        const bool upa = isL ? upLa : upRa, upb = isL ? upLb : upRb;
        const int na = isL ? la : ra, nb = isL ? lb : rb;
        // the side's cotangent on its (na x Mb) grid: pass 4a's result, or A itself
        const double* src = upb ? (isL ? UL + f * 5 * uL : UR + f * 5 * uR) : (isL ? AL + f * 5 * nfl : AR + f * 5 * nfr);
        const int nsrc = upb ? na * Mb : na * nb;
        if (upa) {
          const double* Pa = isL ? PaL : PaR;
          for (int a = 0; a < na; ++a) {
            const double w = __ldg(Pa + a * Ma + m0);
            for (int v = 0; v < 5; ++v) acc[v] += w * src[v * nsrc + a + na * m1];
          }
        } else {
          for (int v = 0; v < 5; ++v) acc[v] += src[v * nsrc + m0 + Ma * m1];
        }
      }
      for (int v = 0; v < 5; ++v) LM[f * 5 * nm + v * nm + x] = acc[v];
    }
    __syncthreads();
    // 5. Roe vector-Jacobian product at the mortar nodes (F* = area Roe), into QL / QR
    for (int t = threadIdx.x; t < cnt * nm; t += blockDim.x) {
      const int f = t / nm, x = t - f * nm;
      double qa[5], qb[5], lf[5], ga[5], gb[5];
      const double area = NR[4 * f + 3];
      for (int v = 0; v < 5; ++v) {
        qa[v] = QL[f * 5 * nm + v * nm + x];
        qb[v] = QR[f * 5 * nm + v * nm + x];
        lf[v] = LM[f * 5 * nm + v * nm + x] * area;
      }
      const double nrm[3] = {NR[4 * f], NR[4 * f + 1], NR[4 * f + 2]};
      roe_vjp<AXIS>(gamma, P.faces[3 * (B.first + f) + 2], qa, qb, nrm, lf, ga, gb);
      for (int v = 0; v < 5; ++v) {
        QL[f * 5 * nm + v * nm + x] = ga[v];
        QR[f * 5 * nm + v * nm + x] = gb[v];
      }
    }
    __syncthreads();
    // 6a. transpose of the xi_b interpolation pass: (Ma x Mb) -> (Ma x nb), into U
    {
      const int nL = upLb ? cnt * Ma * lb : 0, nR = upRb ? cnt * Ma * rb : 0;
      for (int t = threadIdx.x; t < nL + nR; t += blockDim.x) {
        const bool isL = t < nL;
        const int tt = isL ? t : t - nL;
        const int nb = isL ? lb : rb, per = Ma * nb;
        const int f = tt / per, x = tt - f * per, m0 = x % Ma, b = x / Ma;
        const double* Ib = isL ? IbL : IbR;
        const double* src = (isL ? QL : QR) + f * 5 * nm;
        double* dst = (isL ? UL + f * 5 * uL : UR + f * 5 * uR) + x;
        double acc[5] = {0, 0, 0, 0, 0};
        for (int m1 = 0; m1 < Mb; ++m1) {
          const double w = __ldg(Ib + m1 * nb + b);
          for (int v = 0; v < 5; ++v) acc[v] += w * src[v * nm + m0 + Ma * m1];
        }
        for (int v = 0; v < 5; ++v) dst[v * per] = acc[v];
      }
    }
    __syncthreads();
    // 6b. transpose of the xi_a interpolation pass onto each side's face grid, into sadj
    for (int t = threadIdx.x; t < cnt * (nfl + nfr); t += blockDim.x) {
      const bool isL = t < cnt * nfl;
      const int tt = isL ? t : t - cnt * nfl;
      const int nf = isL ? nfl : nfr, na = isL ? la : ra, nb = isL ? lb : rb;
      const int f = tt / nf, x = tt - f * nf, a = x % na, b = x / na;
      const bool upa = isL ? upLa : upRa, upb = isL ? upLb : upRb;
      // the cotangent on the (Ma x nb) grid: pass 6a's result, or the mortar's own
      const double* src = upb ? (isL ? UL + f * 5 * uL : UR + f * 5 * uR) : (isL ? QL : QR) + f * 5 * nm;
      const int nsrc = upb ? Ma * nb : nm;
      double out[5];
      if (upa) {
        const double* Ia = isL ? IaL : IaR;
        for (int v = 0; v < 5; ++v) out[v] = 0.0;
        for (int m0 = 0; m0 < Ma; ++m0) {
          const double w = __ldg(Ia + m0 * na + a);
          for (int v = 0; v < 5; ++v) out[v] += w * src[v * nsrc + m0 + Ma * b];
        }
      } else {
        for (int v = 0; v < 5; ++v) out[v] = src[v * nsrc + a + na * b];
      }
      const int* fr = P.faces + 3 * (B.first + f);
      const int e = isL ? fr[0] : fr[1], dir = fr[2];
      int n1, n2, n3;
      orders_of(m, e, n1, n2, n3);
      double* dst = sadj + 5 * (m.soff[e] + face_offset(n1, n2, n3, isL ? 2 * dir + 1 : 2 * dir)) + x;
      for (int v = 0; v < 5; ++v) dst[v * nf] = out[v];
    }
    __syncthreads();
  }
}

// The general mortars (curved or Navier-Stokes) reversed.  MODE 0 / 1: the
// flux pass; each side's face cotangent (the lift's -/+ (1/w_end)(1/J) v)
// goes back through its own L2 projection to the mortar, then through the
// side's Roe flux with its own normal and, for Navier-Stokes, through the
// BR1 average of both viscous fluxes, to cotangents of both states (and
// gradients) on the mortar grid, and through the transposed interpolation to
// each side's trace nodes: written to sadj (and gadj).  MODE 2: the q-hat
// pass; each side's cotangent of q-hat J a^dir (lS) back to the mortar, then
// to q-hat and half to each trace: added to sadj.
template <int MODE>
struct GMortarAdj {
  static constexpr int nin = GMortar<MODE == 2 ? 0 : MODE>::nin;       // traces (q [, gradient], J a)
  static constexpr int nq = GMortar<MODE == 2 ? 0 : MODE>::nq;         // the cotangent fields sent back
  static constexpr int nout = MODE == 2 ? 15 : 5;                      // the side's output cotangent
  static constexpr int nmid = nin > nout ? nin : nout;
};

template <int MODE>
__host__ __device__ inline size_t mortar_general_adj_smem(const MortarBatch& B) {
  typedef GMortarAdj<MODE> G;
  const int la = B.la, lb = B.lb, ra = B.ra, rb = B.rb;
  const int Ma = la > ra ? la : ra, Mb = lb > rb ? lb : rb, nm = Ma * Mb;
  const int uL = (Ma * lb > la * Mb ? Ma * lb : la * Mb), uR = (Ma * rb > ra * Mb ? Ma * rb : ra * Mb);
  return (size_t)B.count * ((size_t)(G::nin + G::nout) * (la * lb + ra * rb + 2 * nm) + (size_t)G::nmid * (uL + uR));
}

__device__ void viscous_vjp(const DevPhys& ph, const double q[5], const double g[15], const double lf[3][5],
                            double gq[5], double gg[15]);

template <bool AFFINE, int MODE>
__global__ void __launch_bounds__(kVolThreads) adj_mortar_general_kernel(MortarParams P, const double* __restrict__ vin,
                                                                         double* __restrict__ sadj,
                                                                         double* __restrict__ gadj) {
  typedef GMortarAdj<MODE> G;
  constexpr int NIN = G::nin, NQ = G::nq, NOUT = G::nout, NMID = G::nmid;
  extern __shared__ double smem[];
  const MeshView& m = P.m;
  const double gamma = m.ph.gamma;
  for (int it = blockIdx.x; it < P.n_batches; it += gridDim.x) {
    const MortarBatch B = P.batches[it];
    if (bad_batch(P, B, mortar_general_adj_smem<MODE>(B))) continue;
    const int la = B.la, lb = B.lb, ra = B.ra, rb = B.rb, cnt = B.count;
    const int Ma = la > ra ? la : ra, Mb = lb > rb ? lb : rb;
    const int nfl = la * lb, nfr = ra * rb, nm = Ma * Mb;
    const bool upLa = la != Ma, upLb = lb != Mb, upRa = ra != Ma, upRb = rb != Mb;
    const int uL = (Ma * lb > la * Mb ? Ma * lb : la * Mb), uR = (Ma * rb > ra * Mb ? Ma * rb : ra * Mb);
    double* TL = smem;                          // [cnt][NIN][nfl] traces and J a
    double* TR = TL + cnt * NIN * nfl;
    double* AL = TR + cnt * NIN * nfr;          // [cnt][NOUT][nfl] each side's output cotangent
    double* AR = AL + cnt * NOUT * nfl;
    double* UL = AR + cnt * NOUT * nfr;         // [cnt][NMID][uL] pass temporaries
    double* UR = UL + cnt * NMID * uL;
    double* QL = UR + cnt * NMID * uR;          // [cnt][NIN][nm] traces on the mortar, then their cotangents
    double* QR = QL + cnt * NIN * nm;
    double* LL = QR + cnt * NIN * nm;           // [cnt][NOUT][nm] each side's output cotangent on the mortar
    double* LR = LL + cnt * NOUT * nm;
    // 1. traces, J a^dir and the output cotangents
    for (int t = threadIdx.x; t < cnt * (nfl + nfr); t += blockDim.x) {
      const bool isL = t < cnt * nfl;
      const int tt = isL ? t : t - cnt * nfl;
      const int nf = isL ? nfl : nfr, na = isL ? la : ra;
      const int f = tt / nf, p = tt - f * nf;
      const int* fr = P.faces + 3 * (B.first + f);
      const int e = isL ? fr[0] : fr[1], dir = fr[2];
      int n1, n2, n3;
      orders_of(m, e, n1, n2, n3);
      const int n = n1 * n2 * n3;
      const int fe = isL ? 2 * dir + 1 : 2 * dir;
      const int vi = face_vidx(n1, n2, n3, fe, p % na, p / na);
      const int64_t o = m.off[e];
      double* T = (isL ? TL + f * NIN * nfl : TR + f * NIN * nfr) + p;
      double* A = (isL ? AL + f * NOUT * nfl : AR + f * NOUT * nfr) + p;
      for (int v = 0; v < 5; ++v) T[v * nf] = P.q[5 * o + v * n + vi];
      if (MODE == 1)
        for (int v = 0; v < 5; ++v)
          for (int c = 0; c < 3; ++c) T[(5 + v * 3 + c) * nf] = P.grad[15 * o + (c * 5 + v) * n + vi];
      double ja[3];
      face_metric<AFFINE>(m, e, n, vi, dir, ja);
      for (int c = 0; c < 3; ++c) T[(NQ + c) * nf] = ja[c];
      if (MODE == 2) {
        const double* ls = vin + 15 * (m.soff[e] + face_offset(n1, n2, n3, fe));
        for (int c = 0; c < 15; ++c) A[c * nf] = ls[c * nf + p];
      } else {
        const int Nd = (dir == 0 ? n1 : dir == 1 ? n2 : n3) - 1;
        const double cf = (isL ? -1.0 : 1.0) * inv_wend(Nd) * metric<AFFINE>(m.metric, e, o, n, vi, 10);
        for (int v = 0; v < 5; ++v) A[v * nf] = cf * vin[5 * o + v * n + vi];
      }
    }
    __syncthreads();
    // 2-3. the traces interpolated up to the mortar, as in the forward kernel
    const double* IaL = P.basis + c_boff.I[la - 1][Ma - 1];
    const double* IaR = P.basis + c_boff.I[ra - 1][Ma - 1];
    const double* IbL = P.basis + c_boff.I[lb - 1][Mb - 1];
    const double* IbR = P.basis + c_boff.I[rb - 1][Mb - 1];
    {
      const int nL = upLa ? cnt * Ma * lb : 0, nR = upRa ? cnt * Ma * rb : 0;
      for (int t = threadIdx.x; t < nL + nR; t += blockDim.x) {
        const bool isL = t < nL;
        const int tt = isL ? t : t - nL;
        const int nb = isL ? lb : rb, na = isL ? la : ra, per = Ma * nb;
        const int f = tt / per, x = tt - f * per, m0 = x % Ma, b = x / Ma;
        const double* src = isL ? TL + f * NIN * nfl : TR + f * NIN * nfr;
        const double* Ia = isL ? IaL : IaR;
        double* dst = (isL ? UL + f * NMID * uL : UR + f * NMID * uR) + x;
        const int nsrc = na * nb;
        double acc[NIN];
        for (int c = 0; c < NIN; ++c) acc[c] = 0.0;
        for (int a = 0; a < na; ++a) {
          const double w = __ldg(Ia + m0 * na + a);
          for (int c = 0; c < NIN; ++c) acc[c] += w * src[c * nsrc + a + na * b];
        }
        for (int c = 0; c < NIN; ++c) dst[c * per] = acc[c];
      }
    }
    __syncthreads();
    for (int t = threadIdx.x; t < 2 * cnt * nm; t += blockDim.x) {
      const bool isL = t < cnt * nm;
      const int tt = isL ? t : t - cnt * nm;
      const int f = tt / nm, x = tt - f * nm, m0 = x % Ma, m1 = x / Ma;
      const bool upa = isL ? upLa : upRa, upb = isL ? upLb : upRb;
      const int nb = isL ? lb : rb;
      const double* src = upa ? (isL ? UL + f * NMID * uL : UR + f * NMID * uR)
                              : (isL ? TL + f * NIN * nfl : TR + f * NIN * nfr);
      const int nsrc = Ma * nb;
      double* dst = (isL ? QL : QR) + f * NIN * nm + x;
      if (upb) {
        const double* Ib = isL ? IbL : IbR;
        double acc[NIN];
        for (int c = 0; c < NIN; ++c) acc[c] = 0.0;
        for (int b = 0; b < nb; ++b) {
          const double w = __ldg(Ib + m1 * nb + b);
          for (int c = 0; c < NIN; ++c) acc[c] += w * src[c * nsrc + m0 + Ma * b];
        }
        for (int c = 0; c < NIN; ++c) dst[c * nm] = acc[c];
      } else {
        for (int c = 0; c < NIN; ++c) dst[c * nm] = src[c * nsrc + m0 + Ma * m1];
      }
    }
    __syncthreads();
    // 4a. each side's cotangent: transpose of the xi_b projection pass, into U
    const double* PaL = P.basis + c_boff.P[Ma - 1][la - 1];
    const double* PaR = P.basis + c_boff.P[Ma - 1][ra - 1];
    const double* PbL = P.basis + c_boff.P[Mb - 1][lb - 1];
    const double* PbR = P.basis + c_boff.P[Mb - 1][rb - 1];
    {
      const int nL = upLb ? cnt * la * Mb : 0, nR = upRb ? cnt * ra * Mb : 0;
      for (int t = threadIdx.x; t < nL + nR; t += blockDim.x) {
        const bool isL = t < nL;
        const int tt = isL ? t : t - nL;
        const int na = isL ? la : ra, nb = isL ? lb : rb, per = na * Mb;
        const int f = tt / per, x = tt - f * per, a = x % na, m1 = x / na;
        const double* Pb = isL ? PbL : PbR;
        const double* src = isL ? AL + f * NOUT * nfl : AR + f * NOUT * nfr;
        double* dst = (isL ? UL + f * NMID * uL : UR + f * NMID * uR) + x;
        const int nsrc = na * nb;
        double acc[NOUT];
        for (int c = 0; c < NOUT; ++c) acc[c] = 0.0;
        for (int b = 0; b < nb; ++b) {
          const double w = __ldg(Pb + b * Mb + m1);
          for (int c = 0; c < NOUT; ++c) acc[c] += w * src[c * nsrc + a + na * b];
        }
        for (int c = 0; c < NOUT; ++c) dst[c * per] = acc[c];
      }
    }
    __syncthreads();
    // 4b. transpose of the xi_a projection pass, each side onto the mortar grid (not summed:
    //     the two sides' outputs differ)
    for (int t = threadIdx.x; t < 2 * cnt * nm; t += blockDim.x) {
      const bool isL = t < cnt * nm;
      const int tt = isL ? t : t - cnt * nm;
      const int f = tt / nm, x = tt - f * nm, m0 = x % Ma, m1 = x / Ma;
      const bool upa = isL ? upLa : upRa, upb = isL ? upLb : upRb;
      const int na = isL ? la : ra, nb = isL ? lb : rb;
      const double* src = upb ? (isL ? UL + f * NMID * uL : UR + f * NMID * uR)
                              : (isL ? AL + f * NOUT * nfl : AR + f * NOUT * nfr);
      const int nsrc = upb ? na * Mb : na * nb;
      double acc[NOUT];
      if (upa) {
        const double* Pa = isL ? PaL : PaR;
        for (int c = 0; c < NOUT; ++c) acc[c] = 0.0;
        for (int a = 0; a < na; ++a) {
          const double w = __ldg(Pa + a * Ma + m0);
          for (int c = 0; c < NOUT; ++c) acc[c] += w * src[c * nsrc + a + na * m1];
        }
      } else {
        for (int c = 0; c < NOUT; ++c) acc[c] = src[c * nsrc + m0 + Ma * m1];
      }
      double* dst = (isL ? LL : LR) + f * NOUT * nm + x;
      for (int c = 0; c < NOUT; ++c) dst[c * nm] = acc[c];
    }
    __syncthreads();
    // 5. the mortar nodes: cotangents of both traces (and gradients), into QL / QR
    for (int t = threadIdx.x; t < cnt * nm; t += blockDim.x) {
      const int f = t / nm, x = t - f * nm;
      double* ql = QL + f * NIN * nm + x;
      double* qr = QR + f * NIN * nm + x;
      const double* ll = LL + f * NOUT * nm + x;
      const double* lr = LR + f * NOUT * nm + x;
      double jl[3], jr[3], da[5], db[5];
      for (int c = 0; c < 3; ++c) {
        jl[c] = ql[(NQ + c) * nm];
        jr[c] = qr[(NQ + c) * nm];
      }
      if (MODE == 2) {
        for (int v = 0; v < 5; ++v) {
          double dh = 0.0;
          for (int c = 0; c < 3; ++c) dh += ll[(v * 3 + c) * nm] * jl[c] + lr[(v * 3 + c) * nm] * jr[c];
          ql[v * nm] = 0.5 * dh;
          qr[v * nm] = 0.5 * dh;
        }
        continue;
      }
      double qa[5], qb[5], lfl[5], lfr[5], ga[5], gb[5];
      for (int v = 0; v < 5; ++v) {
        qa[v] = ql[v * nm];
        qb[v] = qr[v * nm];
      }
      double nl[3], nr[3];
      const double al = unit_normal(jl, nl), ar = unit_normal(jr, nr);
      for (int v = 0; v < 5; ++v) {
        lfl[v] = al * ll[v * nm];
        lfr[v] = ar * lr[v * nm];
      }
      roe_vjp<false>(gamma, 0, qa, qb, nl, lfl, da, db);
      roe_vjp<false>(gamma, 0, qa, qb, nr, lfr, ga, gb);
      for (int v = 0; v < 5; ++v) {
        da[v] += ga[v];
        db[v] += gb[v];
      }
      if (MODE == 1) {
        double lv[3][5], g[15], vq[5], vg[15];
        for (int d = 0; d < 3; ++d)
          for (int v = 0; v < 5; ++v) lv[d][v] = v >= 1 ? -0.5 * (ll[v * nm] * jl[d] + lr[v * nm] * jr[d]) : 0.0;
        for (int c = 0; c < 15; ++c) g[c] = ql[(5 + c) * nm];
        viscous_vjp(m.ph, qa, g, lv, vq, vg);
        for (int v = 0; v < 5; ++v) da[v] += vq[v];
        for (int c = 0; c < 15; ++c) ql[(5 + c) * nm] = vg[c];
        for (int c = 0; c < 15; ++c) g[c] = qr[(5 + c) * nm];
        viscous_vjp(m.ph, qb, g, lv, vq, vg);
        for (int v = 0; v < 5; ++v) db[v] += vq[v];
        for (int c = 0; c < 15; ++c) qr[(5 + c) * nm] = vg[c];
      }
      for (int v = 0; v < 5; ++v) {
        ql[v * nm] = da[v];
        qr[v * nm] = db[v];
      }
    }
    __syncthreads();
    // 6a. transpose of the xi_b interpolation pass: (Ma x Mb) -> (Ma x nb), into U
    {
      const int nL = upLb ? cnt * Ma * lb : 0, nR = upRb ? cnt * Ma * rb : 0;
      for (int t = threadIdx.x; t < nL + nR; t += blockDim.x) {
        const bool isL = t < nL;
        const int tt = isL ? t : t - nL;
        const int nb = isL ? lb : rb, per = Ma * nb;
        const int f = tt / per, x = tt - f * per, m0 = x % Ma, b = x / Ma;
        const double* Ib = isL ? IbL : IbR;
        const double* src = (isL ? QL : QR) + f * NIN * nm;
        double* dst = (isL ? UL + f * NMID * uL : UR + f * NMID * uR) + x;
        double acc[NQ];
        for (int c = 0; c < NQ; ++c) acc[c] = 0.0;
        for (int m1 = 0; m1 < Mb; ++m1) {
          const double w = __ldg(Ib + m1 * nb + b);
          for (int c = 0; c < NQ; ++c) acc[c] += w * src[c * nm + m0 + Ma * m1];
        }
        for (int c = 0; c < NQ; ++c) dst[c * per] = acc[c];
      }
    }
    __syncthreads();
    // 6b. transpose of the xi_a interpolation pass onto each side's face grid; store
    for (int t = threadIdx.x; t < cnt * (nfl + nfr); t += blockDim.x) {
      const bool isL = t < cnt * nfl;
      const int tt = isL ? t : t - cnt * nfl;
      const int nf = isL ? nfl : nfr, na = isL ? la : ra, nb = isL ? lb : rb;
      const int f = tt / nf, x = tt - f * nf, a = x % na, b = x / na;
      const bool upa = isL ? upLa : upRa, upb = isL ? upLb : upRb;
      const double* src = upb ? (isL ? UL + f * NMID * uL : UR + f * NMID * uR) : (isL ? QL : QR) + f * NIN * nm;
      const int nsrc = upb ? Ma * nb : nm;
      double out[NQ];
      if (upa) {
        const double* Ia = isL ? IaL : IaR;
        for (int c = 0; c < NQ; ++c) out[c] = 0.0;
        for (int m0 = 0; m0 < Ma; ++m0) {
          const double w = __ldg(Ia + m0 * na + a);
          for (int c = 0; c < NQ; ++c) out[c] += w * src[c * nsrc + m0 + Ma * b];
        }
      } else {
        for (int c = 0; c < NQ; ++c) out[c] = src[c * nsrc + a + na * b];
      }
      const int* fr = P.faces + 3 * (B.first + f);
      const int e = isL ? fr[0] : fr[1], dir = fr[2];
      int n1, n2, n3;
      orders_of(m, e, n1, n2, n3);
      const int64_t fo = m.soff[e] + face_offset(n1, n2, n3, isL ? 2 * dir + 1 : 2 * dir);
      if (MODE == 2) {
        for (int v = 0; v < 5; ++v) sadj[5 * fo + v * nf + x] += out[v];
      } else {
        for (int v = 0; v < 5; ++v) sadj[5 * fo + v * nf + x] = out[v];
        if (MODE == 1)
          for (int c = 0; c < 15; ++c) gadj[15 * fo + c * nf + x] = out[5 + c];
      }
    }
    __syncthreads();
  }
}

// The viscous flux of viscous() on any scalar type (Dual for Jacobian
// columns in q or in the gradient g = [v][c]).
template <typename S>
__device__ void viscous_s(const DevPhys& ph, const S q[5], const S g[15], S fv[3][5]) {
  const double gm1 = ph.gamma - 1.0;
  const S ir = 1.0 / q[0];
  const S u[3] = {q[1] * ir, q[2] * ir, q[3] * ir};
  const S p = gm1 * (q[4] - 0.5 * (q[1] * u[0] + q[2] * u[1] + q[3] * u[2]));
  const S pir = p * ir;
  S du[3][3], dT[3];
  const S half_u2 = 0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]);
  for (int c = 0; c < 3; ++c) {
    for (int i = 0; i < 3; ++i) du[i][c] = (g[(1 + i) * 3 + c] - u[i] * g[c]) * ir;
    const S dpc = gm1 * (g[12 + c] - (u[0] * g[3 + c] + u[1] * g[6 + c] + u[2] * g[9 + c]) + half_u2 * g[c]);
    dT[c] = (dpc - pir * g[c]) * ir;
  }
  const S div = du[0][0] + du[1][1] + du[2][2];
  for (int d = 0; d < 3; ++d) {
    S tau[3];
    for (int i = 0; i < 3; ++i) {
      tau[i] = ph.mu * (du[i][d] + du[d][i]);
      if (i == d) tau[i] -= (2.0 / 3.0) * ph.mu * div;
    }
    fv[d][0] = q[0] * 0.0;
    fv[d][1] = tau[0];
    fv[d][2] = tau[1];
    fv[d][3] = tau[2];
    fv[d][4] = u[0] * tau[0] + u[1] * tau[1] + u[2] * tau[2] + ph.kappa_R * dT[d];
  }
}

template <typename S>
__device__ __forceinline__ void bc_ghost_t(const DevPhys& ph, int tag, const S qi[5], S qg[5]) {
  if (tag == DG_BC_WALL) {
    qg[0] = qi[0]; qg[1] = -qi[1]; qg[2] = -qi[2]; qg[3] = -qi[3]; qg[4] = qi[4];
  } else {
    for (int v = 0; v < 5; ++v) qg[v] = qi[v] * 0.0 + ph.qinf[v];
  }
}

template <typename S>
__device__ __forceinline__ void bc_qhat_t(const DevPhys& ph, int tag, const S qi[5], S qh[5]) {
  if (tag == DG_BC_WALL) {
    qh[0] = qi[0]; qh[1] = qi[0] * 0.0; qh[2] = qh[1]; qh[3] = qh[1];
    qh[4] = qi[4] - 0.5 * (qi[1] * qi[1] + qi[2] * qi[2] + qi[3] * qi[3]) / qi[0];
  } else {
    for (int v = 0; v < 5; ++v) qh[v] = qi[v] * 0.0 + ph.qinf[v];
  }
}

// (d fv/d q)^T lf -> gq[5] and (d fv/d g)^T lf -> gg[15] at one node, for
// the viscous flux contracted as sum_d sum_v lf[d][v] fv[d][v]
__device__ void viscous_vjp(const DevPhys& ph, const double q[5], const double g[15], const double lf[3][5],
                            double gq[5], double gg[15]) {
  for (int k = 0; k < 20; ++k) {
    Dual qd[5], gd[15], fd[3][5];
    for (int v = 0; v < 5; ++v) qd[v] = {q[v], k == v ? 1.0 : 0.0};
    for (int c = 0; c < 15; ++c) gd[c] = {g[c], k == 5 + c ? 1.0 : 0.0};
    viscous_s(ph, qd, gd, fd);
    double a = 0.0;
    for (int d = 0; d < 3; ++d)
      for (int v = 0; v < 5; ++v) a += fd[d][v].d * lf[d][v];
    if (k < 5) gq[k] = a;
    else gg[k - 5] = a;
  }
}

// Faces of the warp-per-face list, reversed (one warp per face): conforming
// interior faces (Navier-Stokes or curved meshes) and boundary faces.  The
// numerical flux F* = |J a| Roe - sum_c {{fv_c}} (J a)_c (BR1 average; a
// boundary uses the interior fv, without its energy part at a wall) takes
// the cotangent lf = sum over the sides of -s (1/w_N) v / J; its Jacobian
// transposes go to the traces (sadj) and, for Navier-Stokes, to the face
// nodes' gradients (gadj, [v][c] per element face node).
template <bool AFFINE, bool AXIS, bool NS>
__global__ void __launch_bounds__(32 * kFaceWarps) adj_face_kernel(FaceParams P, const double* __restrict__ vin,
                                                                    double* __restrict__ sadj,
                                                                    double* __restrict__ gadj, double* qinf_adj,
                                                                    const double* scale) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int fidx = blockIdx.x * kFaceWarps + warp;
  if (fidx >= P.n_faces) return;
  const FaceRec fr = P.faces[fidx];
  if (bad_face(P.m, fr)) return;
  const MeshView& m = P.m;
  const double gamma = m.ph.gamma;
  if (fr.kind == 2) {
    const int e = fr.L, f = fr.face, tag = fr.R, dir = f >> 1, side = f & 1;
    int n1, n2, n3;
    orders_of(m, e, n1, n2, n3);
    const int n = n1 * n2 * n3;
    const int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3, nf = na * nb;
    const int64_t o = m.off[e];
    const int Nd = (dir == 0 ? n1 : dir == 1 ? n2 : n3) - 1;
    double* out = sadj + 5 * (m.soff[e] + face_offset(n1, n2, n3, f));
    double* gout = NS ? gadj + 15 * (m.soff[e] + face_offset(n1, n2, n3, f)) : nullptr;
    for (int p = lane; p < nf; p += 32) {
      const int vi = face_vidx(n1, n2, n3, f, p % na, p / na);
      double ja[3], nrm[3];
      face_metric<AFFINE>(m, e, n, vi, dir, ja);
      const double area = unit_normal(ja, nrm);
      const double iJ = metric<AFFINE>(m.metric, e, o, n, vi, 10);
      double qi[5], lf[5], gq[5];
      for (int v = 0; v < 5; ++v) {
        qi[v] = P.q[5 * o + v * n + vi];
        lf[v] = (side ? -1.0 : 1.0) * inv_wend(Nd) * iJ * vin[5 * o + v * n + vi];
      }
      for (int k = 0; k < 5; ++k) {   // Roe against the ghost (which depends on qi at a wall)
        Dual a[5], b[5], F[5];
        for (int v = 0; v < 5; ++v) a[v] = {qi[v], k == v ? 1.0 : 0.0};
        bc_ghost_t(m.ph, tag, a, b);
        if (side) roe_face_d<AXIS>(gamma, dir, a, b, nrm, F);
        else roe_face_d<AXIS>(gamma, dir, b, a, nrm, F);
        double s = 0.0;
        for (int v = 0; v < 5; ++v) s += F[v].d * lf[v];
        gq[k] = area * s;
      }
      if (qinf_adj && tag != DG_BC_WALL) {   // the far-field state is the ghost: its cotangent too
        const double sc = scale ? *scale : 1.0;
        for (int k = 0; k < 5; ++k) {
          Dual a[5], b[5], F[5];
          for (int v = 0; v < 5; ++v) {
            a[v] = {qi[v], 0.0};
            b[v] = {m.ph.qinf[v], k == v ? 1.0 : 0.0};
          }
          if (side) roe_face_d<AXIS>(gamma, dir, a, b, nrm, F);
          else roe_face_d<AXIS>(gamma, dir, b, a, nrm, F);
          double s = 0.0;
          for (int v = 0; v < 5; ++v) s += F[v].d * lf[v];
          atomicAdd(qinf_adj + k, sc * area * s);
        }
      }
      if (NS) {
        double g[15], lv[3][5], vq[5], vg[15];
        for (int v = 0; v < 5; ++v)
          for (int c = 0; c < 3; ++c) g[v * 3 + c] = P.grad[15 * o + (c * 5 + v) * n + vi];
        for (int d = 0; d < 3; ++d)
          for (int v = 0; v < 5; ++v) lv[d][v] = (v >= 1 && (v < 4 || tag != DG_BC_WALL)) ? -ja[d] * lf[v] : 0.0;
        viscous_vjp(m.ph, qi, g, lv, vq, vg);
        for (int v = 0; v < 5; ++v) gq[v] += vq[v];
        for (int v = 0; v < 5; ++v)
          for (int c = 0; c < 3; ++c) gout[(v * 3 + c) * nf + p] = vg[v * 3 + c];
      }
      for (int v = 0; v < 5; ++v) out[v * nf + p] = gq[v];
    }
    return;
  }
  if (fr.kind != 0) return;   // p-nonconforming faces run in the mortar batches
  const int L = fr.L, R = fr.R, dir = fr.face;
  int l1, l2, l3, r1, r2, r3;
  orders_of(m, L, l1, l2, l3);
  orders_of(m, R, r1, r2, r3);
  const int nL = l1 * l2 * l3, nR = r1 * r2 * r3;
  const int64_t oL = m.off[L], oR = m.off[R];
  const int fL = 2 * dir + 1, fR = 2 * dir;
  const int la = dir == 0 ? l2 : l1, lb = dir == 2 ? l2 : l3, nf = la * lb;
  const int NdL = (dir == 0 ? l1 : dir == 1 ? l2 : l3) - 1, NdR = (dir == 0 ? r1 : dir == 1 ? r2 : r3) - 1;
  double* outL = sadj + 5 * (m.soff[L] + face_offset(l1, l2, l3, fL));
  double* outR = sadj + 5 * (m.soff[R] + face_offset(r1, r2, r3, fR));
  for (int p = lane; p < nf; p += 32) {
    const int a = p % la, b = p / la;
    const int iL = face_vidx(l1, l2, l3, fL, a, b), iR = face_vidx(r1, r2, r3, fR, a, b);
    double ja[3], nrm[3];
    face_metric<AFFINE>(m, L, nL, iL, dir, ja);
    const double area = unit_normal(ja, nrm);
    const double iJL = metric<AFFINE>(m.metric, L, oL, nL, iL, 10), iJR = metric<AFFINE>(m.metric, R, oR, nR, iR, 10);
    double qL[5], qR[5], lf[5], gL[5], gR[5];
    for (int v = 0; v < 5; ++v) {
      qL[v] = P.q[5 * oL + v * nL + iL];
      qR[v] = P.q[5 * oR + v * nR + iR];
      lf[v] = -inv_wend(NdL) * iJL * vin[5 * oL + v * nL + iL] + inv_wend(NdR) * iJR * vin[5 * oR + v * nR + iR];
    }
    double lfa[5];
    for (int v = 0; v < 5; ++v) lfa[v] = area * lf[v];
    roe_vjp<AXIS>(gamma, dir, qL, qR, nrm, lfa, gL, gR);
    if (NS) {
      double gg[15], lv[3][5], vq[5], vg[15];
      for (int d = 0; d < 3; ++d)
        for (int v = 0; v < 5; ++v) lv[d][v] = v >= 1 ? -0.5 * ja[d] * lf[v] : 0.0;
      for (int s2 = 0; s2 < 2; ++s2) {
        const int e = s2 ? R : L, vi = s2 ? iR : iL, ne = s2 ? nR : nL;
        const int64_t oe = s2 ? oR : oL;
        const double* qe = s2 ? qR : qL;
        for (int v = 0; v < 5; ++v)
          for (int c = 0; c < 3; ++c) gg[v * 3 + c] = P.grad[15 * oe + (c * 5 + v) * ne + vi];
        viscous_vjp(m.ph, qe, gg, lv, vq, vg);
        double* gq = s2 ? gR : gL;
        for (int v = 0; v < 5; ++v) gq[v] += vq[v];
        int e1, e2, e3;
        orders_of(m, e, e1, e2, e3);
        double* go = gadj + 15 * (m.soff[e] + face_offset(e1, e2, e3, s2 ? fR : fL));
        for (int v = 0; v < 5; ++v)
          for (int c = 0; c < 3; ++c) go[(v * 3 + c) * nf + p] = vg[v * 3 + c];
      }
    }
    for (int v = 0; v < 5; ++v) {
      outL[v * nf + p] = gL[v];
      outR[v * nf + p] = gR[v];
    }
  }
}

// q-hat of BR1, reversed (one warp per face): the cotangent of each side's
// lifted q-hat J a^dir (lS, [v][c] per element face node) becomes that of
// q-hat, then of the traces: half to each side of an interior face, through
// q-hat(q_in) at a wall, nothing at the far field (q-hat = q_inf).  Added to
// sadj.
template <bool AFFINE>
__global__ void __launch_bounds__(32 * kFaceWarps) adj_qhat_kernel(FaceParams P, const double* __restrict__ lS,
                                                                    double* __restrict__ sadj, double* qinf_adj,
                                                                    const double* scale) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int fidx = blockIdx.x * kFaceWarps + warp;
  if (fidx >= P.n_faces) return;
  const FaceRec fr = P.faces[fidx];
  if (bad_face(P.m, fr)) return;
  const MeshView& m = P.m;
  if (fr.kind == 2) {
    const int e = fr.L, f = fr.face, tag = fr.R, dir = f >> 1;
    if (tag != DG_BC_WALL && !qinf_adj) return;
    int n1, n2, n3;
    orders_of(m, e, n1, n2, n3);
    const int n = n1 * n2 * n3;
    const int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3, nf = na * nb;
    const int64_t o = m.off[e];
    const int64_t fo = m.soff[e] + face_offset(n1, n2, n3, f);
    for (int p = lane; p < nf; p += 32) {
      const int vi = face_vidx(n1, n2, n3, f, p % na, p / na);
      double ja[3], lh[5];
      face_metric<AFFINE>(m, e, n, vi, dir, ja);
      for (int v = 0; v < 5; ++v) {
        lh[v] = 0.0;
        for (int c = 0; c < 3; ++c) lh[v] += ja[c] * lS[15 * fo + (v * 3 + c) * nf + p];
      }
      if (tag != DG_BC_WALL) {   // far field: q-hat = q_inf
        const double sc = scale ? *scale : 1.0;
        for (int v = 0; v < 5; ++v) atomicAdd(qinf_adj + v, sc * lh[v]);
        continue;
      }
      for (int k = 0; k < 5; ++k) {
        Dual qi[5], qh[5];
        for (int v = 0; v < 5; ++v) qi[v] = {P.q[5 * o + v * n + vi], k == v ? 1.0 : 0.0};
        bc_qhat_t(m.ph, tag, qi, qh);
        double s = 0.0;
        for (int v = 0; v < 5; ++v) s += qh[v].d * lh[v];
        sadj[5 * fo + k * nf + p] += s;
      }
    }
    return;
  }
  if (fr.kind != 0) return;
  const int L = fr.L, R = fr.R, dir = fr.face;
  int l1, l2, l3, r1, r2, r3;
  orders_of(m, L, l1, l2, l3);
  orders_of(m, R, r1, r2, r3);
  const int nL = l1 * l2 * l3;
  const int la = dir == 0 ? l2 : l1, lb = dir == 2 ? l2 : l3, nf = la * lb;
  const int64_t foL = m.soff[L] + face_offset(l1, l2, l3, 2 * dir + 1);
  const int64_t foR = m.soff[R] + face_offset(r1, r2, r3, 2 * dir);
  for (int p = lane; p < nf; p += 32) {
    const int iL = face_vidx(l1, l2, l3, 2 * dir + 1, p % la, p / la);
    double ja[3];
    face_metric<AFFINE>(m, L, nL, iL, dir, ja);   // both sides lift q-hat J a^dir with L's metric
    for (int v = 0; v < 5; ++v) {
      double lh = 0.0;
      for (int c = 0; c < 3; ++c)
        lh += ja[c] * (lS[15 * foL + (v * 3 + c) * nf + p] + lS[15 * foR + (v * 3 + c) * nf + p]);
      sadj[5 * foL + v * nf + p] += 0.5 * lh;
      sadj[5 * foR + v * nf + p] += 0.5 * lh;
    }
  }
}

struct AdjParams {
  MeshView m;
  const WorkItem* items;
  const int32_t* elist;
  const int32_t* ilist;
  int n_items;
  int n_items_all;         // length of items
  const double* q;
  const double* grad;      // BR1 gradient of q (Navier-Stokes)
  const double* v;         // cotangent of the residual (state layout)
  const double* sadj;      // trace cotangents per element face node (face-buffer layout), or null
  const double* gadj;      // gradient cotangents per element face node [v][c] (Navier-Stokes)
  double* gout;            // the gradient's cotangent, gradient layout (Navier-Stokes)
  double* lS;              // cotangent of the lifted q-hat J a^dir per element face node [v][c]
  double* out;             // J^T v, or out += (*scale) J^T v
  const double* scale;     // device scalar (accumulate mode)
  int accumulate;
  const double* basis;
};

// Volume part, reversed, one tile per CTA: u = -v/J; the transposed GL
// derivatives lF_i = D_i^T u; the inner-flux part of the lift, lF_dir -=
// s (1/w_N) u at each face's nodes; then per node mu_d = sum_i J a^i_d lF_i
// and J^T v = sum_d (d phi_d / d q)^T mu_d with phi_d = f_d - fv_d (five Dual
// evaluations of the Euler flux; Navier-Stokes adds the viscous flux's
// columns in q and, into gout, in the gradient).  With sadj, the trace
// cotangents of the node's faces are added here.
template <bool AFFINE, bool AXIS, bool NS>
__global__ void __launch_bounds__(kVolThreads) adj_volume_kernel(AdjParams P) {
  extern __shared__ double smem[];
  const MeshView& m = P.m;
  const double gm1 = m.ph.gamma - 1.0;
  for (int it = blockIdx.x; it < P.n_items; it += gridDim.x) {
    WorkItem w;
    if (!take_item(P.m, P.items, P.ilist ? P.ilist[it] : it, P.n_items_all, P.elist, 20, w)) continue;
    const int n1 = w.n1 + 1, n2 = w.n2 + 1, n3 = w.n3 + 1, n = n1 * n2 * n3;
    const int slots = w.count * n;
    double* U = smem;                                 // [count][5][n]
    double* LF = smem + (size_t)w.count * 5 * n;      // [count][3][5][n]
    for (int s = threadIdx.x; s < slots; s += blockDim.x) {
      const int el = s / n, p = s - el * n;
      const int e = P.elist[w.first + el];
      const int64_t o = m.off[e];
      const double iJ = metric<AFFINE>(m.metric, e, o, n, p, 10);
      for (int v = 0; v < 5; ++v) U[(size_t)el * 5 * n + v * n + p] = -P.v[5 * o + v * n + p] * iJ;
    }
    __syncthreads();
    const double* D1 = P.basis + c_boff.D[w.n1];
    const double* D2 = P.basis + c_boff.D[w.n2];
    const double* D3 = P.basis + c_boff.D[w.n3];
    for (int s = threadIdx.x; s < slots; s += blockDim.x) {
      const int el = s / n, p = s - el * n;
      const int i = p % n1, j = (p / n1) % n2, k = p / (n1 * n2);
      const double* Ue = U + (size_t)el * 5 * n;
      double* L = LF + (size_t)el * 15 * n;
      double acc[5];
      for (int v = 0; v < 5; ++v) acc[v] = 0.0;
      for (int mm = 0; mm < n1; ++mm) {
        const double d = __ldg(D1 + mm * n1 + i);
        for (int v = 0; v < 5; ++v) acc[v] += d * Ue[v * n + mm + n1 * (j + n2 * k)];
      }
      for (int v = 0; v < 5; ++v) L[v * n + p] = acc[v];
      for (int v = 0; v < 5; ++v) acc[v] = 0.0;
      for (int mm = 0; mm < n2; ++mm) {
        const double d = __ldg(D2 + mm * n2 + j);
        for (int v = 0; v < 5; ++v) acc[v] += d * Ue[v * n + i + n1 * (mm + n2 * k)];
      }
      for (int v = 0; v < 5; ++v) L[(5 + v) * n + p] = acc[v];
      for (int v = 0; v < 5; ++v) acc[v] = 0.0;
      for (int mm = 0; mm < n3; ++mm) {
        const double d = __ldg(D3 + mm * n3 + k);
        for (int v = 0; v < 5; ++v) acc[v] += d * Ue[v * n + i + n1 * (j + n2 * mm)];
      }
      for (int v = 0; v < 5; ++v) L[(10 + v) * n + p] = acc[v];
    }
    __syncthreads();
    // the inner flux in the lift: the two faces of a direction touch
    // disjoint nodes and each direction its own lF, so one pass has no races
    for (int dir = 0; dir < 3; ++dir) {
      const int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3, fsz = na * nb;
      const int Nd = dir == 0 ? w.n1 : (dir == 1 ? w.n2 : w.n3);
      const double iw = inv_wend(Nd);
      const int per_el = 2 * fsz;
      for (int s = threadIdx.x; s < w.count * per_el; s += blockDim.x) {
        const int el = s / per_el, r = s - el * per_el;
        const int side = r / fsz, fn = r - side * fsz;
        const int p = face_vidx(n1, n2, n3, 2 * dir + side, fn % na, fn / na);
        const double sg = side ? iw : -iw;
        for (int v = 0; v < 5; ++v)
          LF[(size_t)el * 15 * n + (dir * 5 + v) * n + p] -= sg * U[(size_t)el * 5 * n + v * n + p];
      }
    }
    __syncthreads();
    for (int s = threadIdx.x; s < slots; s += blockDim.x) {
      const int el = s / n, p = s - el * n;
      const int e = P.elist[w.first + el];
      const int64_t o = m.off[e];
      const double* L = LF + (size_t)el * 15 * n;
      double mu[3][5];
      for (int d = 0; d < 3; ++d)
        for (int v = 0; v < 5; ++v) {
          if (AXIS) {
            mu[d][v] = metric<AFFINE>(m.metric, e, o, n, p, 4 * d) * L[(d * 5 + v) * n + p];
          } else {
            mu[d][v] = 0.0;
            for (int i = 0; i < 3; ++i)
              mu[d][v] += metric<AFFINE>(m.metric, e, o, n, p, 3 * i + d) * L[(i * 5 + v) * n + p];
          }
        }
      double q[5], lam[5];
      for (int v = 0; v < 5; ++v) q[v] = P.q[5 * o + v * n + p];
      for (int kk = 0; kk < 5; ++kk) {
        Dual qd[5], fd[3][5];
        for (int v = 0; v < 5; ++v) qd[v] = {q[v], kk == v ? 1.0 : 0.0};
        euler_flux3(gm1, qd, fd);
        double g = 0.0;
        for (int d = 0; d < 3; ++d)
          for (int v = 0; v < 5; ++v) g += fd[d][v].d * mu[d][v];
        lam[kk] = g;
      }
      if (NS) {   // phi = f - fv: the viscous columns with the opposite sign
        double g[15], lv[3][5], vq[5], vg[15];
        for (int v = 0; v < 5; ++v)
          for (int c = 0; c < 3; ++c) g[v * 3 + c] = P.grad[15 * o + (c * 5 + v) * n + p];
        for (int d = 0; d < 3; ++d)
          for (int v = 0; v < 5; ++v) lv[d][v] = -mu[d][v];
        viscous_vjp(m.ph, q, g, lv, vq, vg);
        for (int v = 0; v < 5; ++v) lam[v] += vq[v];
        for (int v = 0; v < 5; ++v)
          for (int c = 0; c < 3; ++c) P.gout[15 * o + (c * 5 + v) * n + p] = vg[v * 3 + c];
      }
      if (P.sadj) {   // trace cotangents of the faces through this node
        const int i = p % n1, j = (p / n1) % n2, k = p / (n1 * n2);
        const double* sb = P.sadj + 5 * m.soff[e];
        for (int f = 0; f < 6; ++f) {
          const int dir = f >> 1, side = f & 1;
          const int c = dir == 0 ? i : dir == 1 ? j : k, nd = dir == 0 ? n1 : dir == 1 ? n2 : n3;
          if (c != (side ? nd - 1 : 0)) continue;
          const int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3, nf = na * nb;
          const int a = dir == 0 ? j : i, b = dir == 2 ? j : k;
          const double* fb = sb + 5 * face_offset(n1, n2, n3, f) + a + na * b;
          for (int v = 0; v < 5; ++v) lam[v] += fb[v * nf];
        }
      }
      if (P.accumulate) {
        const double sc = *P.scale;
        for (int v = 0; v < 5; ++v) P.out[5 * o + v * n + p] += sc * lam[v];
      } else {
        for (int v = 0; v < 5; ++v) P.out[5 * o + v * n + p] = lam[v];
      }
    }
    __syncthreads();
  }
}

// The BR1 gradient, reversed, one tile per CTA.  Forward, per component c:
// g_c = (1/J) [sum_i D_i (J a^i_c q) + sum over the node's faces s (1/w_N)
// (qhat J a^dir_c - J a^dir_c q)].  With gamma_c = (gout_c + the node's
// face cotangents gadj) / J: out += sum_c sum_i J a^i_c D_i^T gamma_c - the
// lift's inner part, and lS (the cotangent of each face node's lifted
// q-hat J a^dir) = s (1/w_N) gamma.
template <bool AFFINE>
__global__ void __launch_bounds__(kVolThreads) adj_gradient_kernel(AdjParams P) {
  extern __shared__ double smem[];
  const MeshView& m = P.m;
  for (int it = blockIdx.x; it < P.n_items; it += gridDim.x) {
    WorkItem w;
    if (!take_item(P.m, P.items, P.ilist ? P.ilist[it] : it, P.n_items_all, P.elist, 15, w)) continue;
    const int n1 = w.n1 + 1, n2 = w.n2 + 1, n3 = w.n3 + 1, n = n1 * n2 * n3;
    const int slots = w.count * n;
    double* Gm = smem;   // [count][3][5][n]: gamma_c[v]
    for (int s = threadIdx.x; s < slots; s += blockDim.x) {
      const int el = s / n, p = s - el * n;
      const int e = P.elist[w.first + el];
      const int64_t o = m.off[e];
      const int i = p % n1, j = (p / n1) % n2, k = p / (n1 * n2);
      double gm[15];
      for (int c = 0; c < 3; ++c)
        for (int v = 0; v < 5; ++v) gm[c * 5 + v] = P.gout[15 * o + (c * 5 + v) * n + p];
      const double* gb = P.gadj + 15 * m.soff[e];
      for (int f = 0; f < 6; ++f) {
        const int dir = f >> 1, side = f & 1;
        const int cc = dir == 0 ? i : dir == 1 ? j : k, nd = dir == 0 ? n1 : dir == 1 ? n2 : n3;
        if (cc != (side ? nd - 1 : 0)) continue;
        const int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3, nf = na * nb;
        const int a = dir == 0 ? j : i, b = dir == 2 ? j : k;
        const double* fb = gb + 15 * face_offset(n1, n2, n3, f) + a + na * b;
        for (int v = 0; v < 5; ++v)
          for (int c = 0; c < 3; ++c) gm[c * 5 + v] += fb[(v * 3 + c) * nf];
      }
      const double iJ = metric<AFFINE>(m.metric, e, o, n, p, 10);
      for (int c = 0; c < 15; ++c) Gm[(size_t)el * 15 * n + c * n + p] = gm[c] * iJ;
    }
    __syncthreads();
    const double* D1 = P.basis + c_boff.D[w.n1];
    const double* D2 = P.basis + c_boff.D[w.n2];
    const double* D3 = P.basis + c_boff.D[w.n3];
    for (int s = threadIdx.x; s < slots; s += blockDim.x) {
      const int el = s / n, p = s - el * n;
      const int e = P.elist[w.first + el];
      const int64_t o = m.off[e];
      const int i = p % n1, j = (p / n1) % n2, k = p / (n1 * n2);
      const double* G = Gm + (size_t)el * 15 * n;
      double lam[5] = {0, 0, 0, 0, 0};
      for (int c = 0; c < 3; ++c) {
        double a1[5] = {0, 0, 0, 0, 0}, a2[5] = {0, 0, 0, 0, 0}, a3[5] = {0, 0, 0, 0, 0};
        for (int mm = 0; mm < n1; ++mm) {
          const double d = __ldg(D1 + mm * n1 + i);
          for (int v = 0; v < 5; ++v) a1[v] += d * G[(c * 5 + v) * n + mm + n1 * (j + n2 * k)];
        }
        for (int mm = 0; mm < n2; ++mm) {
          const double d = __ldg(D2 + mm * n2 + j);
          for (int v = 0; v < 5; ++v) a2[v] += d * G[(c * 5 + v) * n + i + n1 * (mm + n2 * k)];
        }
        for (int mm = 0; mm < n3; ++mm) {
          const double d = __ldg(D3 + mm * n3 + k);
          for (int v = 0; v < 5; ++v) a3[v] += d * G[(c * 5 + v) * n + i + n1 * (j + n2 * mm)];
        }
        const double j1 = metric<AFFINE>(m.metric, e, o, n, p, c), j2 = metric<AFFINE>(m.metric, e, o, n, p, 3 + c),
                     j3 = metric<AFFINE>(m.metric, e, o, n, p, 6 + c);
        for (int v = 0; v < 5; ++v) lam[v] += j1 * a1[v] + j2 * a2[v] + j3 * a3[v];
      }
      // the lift: inner part on q, face part on the lifted q-hat
      double* lb_ = P.lS + 15 * m.soff[e];
      for (int f = 0; f < 6; ++f) {
        const int dir = f >> 1, side = f & 1;
        const int cc = dir == 0 ? i : dir == 1 ? j : k, nd = dir == 0 ? n1 : dir == 1 ? n2 : n3;
        if (cc != (side ? nd - 1 : 0)) continue;
        const int Nd = nd - 1;
        const double sg = (side ? 1.0 : -1.0) * inv_wend(Nd);
        const int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3, nf = na * nb;
        const int a = dir == 0 ? j : i, b = dir == 2 ? j : k;
        double* fb = lb_ + 15 * face_offset(n1, n2, n3, f) + a + na * b;
        for (int c = 0; c < 3; ++c) {
          const double jd = metric<AFFINE>(m.metric, e, o, n, p, 3 * dir + c);
          for (int v = 0; v < 5; ++v) {
            lam[v] -= sg * jd * G[(c * 5 + v) * n + p];
            fb[(v * 3 + c) * nf] = sg * G[(c * 5 + v) * n + p];
          }
        }
      }
      for (int v = 0; v < 5; ++v) P.out[5 * o + v * n + p] += lam[v];
    }
    __syncthreads();
  }
}

// out += the trace cotangents of each node's faces (sadj), one tile per CTA
__global__ void __launch_bounds__(kVolThreads) adj_gather_kernel(AdjParams P) {
  const MeshView& m = P.m;
  for (int it = blockIdx.x; it < P.n_items; it += gridDim.x) {
    WorkItem w;
    if (!take_item(P.m, P.items, P.ilist ? P.ilist[it] : it, P.n_items_all, P.elist, 0, w)) continue;
    const int n1 = w.n1 + 1, n2 = w.n2 + 1, n3 = w.n3 + 1, n = n1 * n2 * n3;
    for (int s = threadIdx.x; s < w.count * n; s += blockDim.x) {
      const int el = s / n, p = s - el * n;
      const int e = P.elist[w.first + el];
      const int64_t o = m.off[e];
      const int i = p % n1, j = (p / n1) % n2, k = p / (n1 * n2);
      const double* sb = P.sadj + 5 * m.soff[e];
      for (int f = 0; f < 6; ++f) {
        const int dir = f >> 1, side = f & 1;
        const int c = dir == 0 ? i : dir == 1 ? j : k, nd = dir == 0 ? n1 : dir == 1 ? n2 : n3;
        if (c != (side ? nd - 1 : 0)) continue;
        const int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3, nf = na * nb;
        const int a = dir == 0 ? j : i, b = dir == 2 ? j : k;
        const double* fb = sb + 5 * face_offset(n1, n2, n3, f) + a + na * b;
        for (int v = 0; v < 5; ++v) P.out[5 * o + v * n + p] += fb[v * nf];
      }
    }
  }
}

// y += (*scale) x
__global__ void axpy_dev_kernel(double* __restrict__ y, const double* __restrict__ x, const double* scale, int64_t n) {
  const double a = *scale;
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] += a * x[i];
}

// y = a y + b x over n values (a = 0: y is not read, so it may hold anything)
__global__ void axpby_kernel(double* __restrict__ y, const double* __restrict__ x, double a, double b, int64_t n) {
  for (int64_t i = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
    y[i] = (a == 0.0 ? 0.0 : a * y[i]) + b * x[i];
}

}  // namespace

// shared memory (doubles) of one mortar batch in the adjoint kernel

namespace dgk {

template <bool AFF, bool AX, bool NSV>
static cudaError_t launch_adj_volume(dg_mesh_impl* m, AdjParams A) {
  cudaError_t err;
  for (auto& c : m->vol_classes) {
    A.ilist = c.d_list;
    A.n_items = c.n;
    const size_t smem = sizeof(double) * 20 * c.S;
    if ((err = allow_smem(adj_volume_kernel<AFF, AX, NSV>, smem))) return err;
    adj_volume_kernel<AFF, AX, NSV><<<c.n, kVolThreads, smem, m->stream>>>(A);
    if ((err = cudaGetLastError())) return err;
  }
  return cudaSuccess;
}

static MortarParams mortar_params(dg_mesh_impl* m, const double* q) {
  MortarParams M{};
  M.m = view(m);
  M.batches = reinterpret_cast<const MortarBatch*>(m->d_mbatches);
  M.n_batches = m->n_mbatches;
  M.n_mfaces = m->n_mfaces;
  M.faces = m->d_mfaces;
  M.q = q;
  M.surf = nullptr;
  M.basis = m->basis64;
  M.grad = m->d_grad;
  return M;
}

#define DG_ADJ_GMORTAR(AFF, MODE, VIN, GADJ)                                                                 \
  {                                                                                                        \
    if ((err = allow_smem(adj_mortar_general_kernel<AFF, MODE>, smem))) return err;                       \
    adj_mortar_general_kernel<AFF, MODE><<<m->n_mbatches, kVolThreads, smem, m->stream>>>(M, VIN, m->d_sadj, \
                                                                                           GADJ);          \
  }

// BR1 q-hat reversed on every face: the listed faces, then the general mortars
static cudaError_t adj_qhat_all(dg_mesh_impl* m, const double* q, double* qinf_adj, const double* scale) {
  cudaError_t err;
  if (m->n_faces) {
    FaceParams F = dgk_face_params_for(m, q, m->d_sadj);
    const int grid = (m->n_faces + kFaceWarps - 1) / kFaceWarps;
    if (m->affine) adj_qhat_kernel<true><<<grid, 32 * kFaceWarps, 0, m->stream>>>(F, m->d_lS, m->d_sadj, qinf_adj, scale);
    else adj_qhat_kernel<false><<<grid, 32 * kFaceWarps, 0, m->stream>>>(F, m->d_lS, m->d_sadj, qinf_adj, scale);
    if ((err = cudaGetLastError())) return err;
  }
  if (m->n_mbatches && m->general_mortars) {
    MortarParams M = mortar_params(m, q);
    const size_t smem = sizeof(double) * mortar_adj_smem_max(m);
    if (m->affine) DG_ADJ_GMORTAR(true, 2, m->d_lS, nullptr) else DG_ADJ_GMORTAR(false, 2, m->d_lS, nullptr)
    if ((err = cudaGetLastError())) return err;
  }
  return cudaSuccess;
}

cudaError_t residual_vjp(dg_mesh_impl* m, const double* q, const double* v, double* out, const double* scale,
                         bool accumulate, double* qinf_adj) {
  cudaError_t err;
  const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
  if (ns) {   // the BR1 gradient of q, as in the forward residual
    if ((err = face_qhat(m, q)) || (err = gradient(m, q, m->d_grad, false))) return err;
  }
  const int nvc = (int)m->vol_classes.size();
  Prof pr(m, DG_KERNEL_ADJOINT,
          (m->n_faces ? 1 : 0) + (m->n_mbatches ? 1 : 0) + nvc +
              (ns ? 2 * nvc + (m->n_faces ? 1 : 0) + (m->n_mbatches && m->general_mortars ? 1 : 0) +
                        (accumulate ? 1 : 0)
                  : 0));
  // 1. faces: warp-per-face list (conforming on curved / Navier-Stokes meshes, boundaries) and mortar batches
  if (m->n_faces) {
    FaceParams F = dgk_face_params_for(m, q, m->d_sadj);
    F.grad = m->d_grad;
    const int grid = (m->n_faces + kFaceWarps - 1) / kFaceWarps;
    if (ns) {
      if (m->affine) adj_face_kernel<true, false, true><<<grid, 32 * kFaceWarps, 0, m->stream>>>(F, v, m->d_sadj, m->d_gadj, qinf_adj, scale);
      else adj_face_kernel<false, false, true><<<grid, 32 * kFaceWarps, 0, m->stream>>>(F, v, m->d_sadj, m->d_gadj, qinf_adj,
                                                                                     scale);
    } else if (m->axis) {
      adj_face_kernel<true, true, false><<<grid, 32 * kFaceWarps, 0, m->stream>>>(F, v, m->d_sadj, nullptr, qinf_adj, scale);
    } else if (m->affine) {
      adj_face_kernel<true, false, false><<<grid, 32 * kFaceWarps, 0, m->stream>>>(F, v, m->d_sadj, nullptr, qinf_adj,
                                                                                   scale);
    } else {
      adj_face_kernel<false, false, false><<<grid, 32 * kFaceWarps, 0, m->stream>>>(F, v, m->d_sadj, nullptr, qinf_adj,
                                                                                    scale);
    }
    if ((err = cudaGetLastError())) return err;
  }
  if (m->n_mbatches && m->general_mortars) {
    MortarParams M = mortar_params(m, q);
    const size_t smem = sizeof(double) * mortar_adj_smem_max(m);
    if (m->affine) {
      if (ns) { DG_ADJ_GMORTAR(true, 1, v, m->d_gadj) } else { DG_ADJ_GMORTAR(true, 0, v, nullptr) }
    } else {
      if (ns) { DG_ADJ_GMORTAR(false, 1, v, m->d_gadj) } else { DG_ADJ_GMORTAR(false, 0, v, nullptr) }
    }
    if ((err = cudaGetLastError())) return err;
  } else if (m->n_mbatches) {
    MortarParams M = mortar_params(m, q);
    const size_t smem = sizeof(double) * mortar_adj_smem_max(m);
    if (m->axis) {
      if ((err = allow_smem(adj_mortar_kernel<true>, smem))) return err;
      adj_mortar_kernel<true><<<m->n_mbatches, kVolThreads, smem, m->stream>>>(M, v, m->d_sadj);
    } else {
      if ((err = allow_smem(adj_mortar_kernel<false>, smem))) return err;
      adj_mortar_kernel<false><<<m->n_mbatches, kVolThreads, smem, m->stream>>>(M, v, m->d_sadj);
    }
    if ((err = cudaGetLastError())) return err;
  }
  AdjParams A;
  memset(&A, 0, sizeof(A));
  A.m = view(m);
  A.items = m->d_vitems;
  A.n_items_all = m->n_vitems;
  A.elist = m->d_velist;
  A.q = q;
  A.grad = m->d_grad;
  A.v = v;
  A.basis = m->basis64;
  if (!ns) {   // 2. volume, with the face cotangents gathered, straight into out
    A.sadj = m->d_sadj;
    A.out = out;
    A.scale = scale;
    A.accumulate = accumulate;
    if (m->axis) return launch_adj_volume<true, true, false>(m, A);
    if (m->affine) return launch_adj_volume<true, false, false>(m, A);
    return launch_adj_volume<false, false, false>(m, A);
  }
  // Navier-Stokes: volume (into the scratch state, and the gradient's
  // cotangent), BR1 gradient reversed, q-hat reversed, the face cotangents
  // gathered, then into out
  double* tmp = m->d_adjt;
  A.sadj = nullptr;
  A.out = tmp;
  A.gout = m->d_lG;
  A.gadj = m->d_gadj;
  A.lS = m->d_lS;
  if ((err = m->affine ? launch_adj_volume<true, false, true>(m, A) : launch_adj_volume<false, false, true>(m, A)))
    return err;
  for (auto& c : m->vol_classes) {
    A.ilist = c.d_list;
    A.n_items = c.n;
    const size_t smem = sizeof(double) * 15 * c.S;
    if (m->affine) {
      if ((err = allow_smem(adj_gradient_kernel<true>, smem))) return err;
      adj_gradient_kernel<true><<<c.n, kVolThreads, smem, m->stream>>>(A);
    } else {
      if ((err = allow_smem(adj_gradient_kernel<false>, smem))) return err;
      adj_gradient_kernel<false><<<c.n, kVolThreads, smem, m->stream>>>(A);
    }
    if ((err = cudaGetLastError())) return err;
  }
  if ((err = adj_qhat_all(m, q, qinf_adj, scale))) return err;
  A.sadj = m->d_sadj;
  for (auto& c : m->vol_classes) {
    A.ilist = c.d_list;
    A.n_items = c.n;
    adj_gather_kernel<<<c.n, kVolThreads, 0, m->stream>>>(A);
    if ((err = cudaGetLastError())) return err;
  }
  const int64_t ns5 = 5 * m->n_nodes;
  if (!accumulate) return cudaMemcpyAsync(out, tmp, sizeof(double) * ns5, cudaMemcpyDeviceToDevice, m->stream);
  const int grid = grid_for((int)std::min<int64_t>((ns5 + 255) / 256, 1 << 20), 8);
  axpy_dev_kernel<<<grid, 256, 0, m->stream>>>(out, tmp, scale, ns5);
  return cudaGetLastError();
}

#undef DG_ADJ_GMORTAR

size_t mortar_adj_smem_max(dg_mesh_impl* m) {
  size_t sm = 0;
  const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
  for (int b = 0; b < m->n_mbatches; ++b) {
    const int32_t* B = &m->h_mbatches[6 * b];
    if (m->general_mortars) {
      const MortarBatch mb{B[0], B[1], B[2], B[3], B[4], B[5]};
      sm = std::max(sm, ns ? std::max(mortar_general_adj_smem<1>(mb), mortar_general_adj_smem<2>(mb))
                           : mortar_general_adj_smem<0>(mb));
    } else {
      sm = std::max(sm, mortar_adj_smem_doubles(B[1], B[2], B[3], B[4], B[5]));
    }
  }
  return sm;
}

cudaError_t axpby(dg_mesh_impl* m, double* y, const double* x, double a, double b, int64_t n) {
  const int grid = grid_for((int)std::min<int64_t>((n + 255) / 256, 1 << 20), 8);
  Prof pr(m, DG_KERNEL_ADJOINT);
  axpby_kernel<<<grid, 256, 0, m->stream>>>(y, x, a, b, n);
  return cudaGetLastError();
}

}  // namespace dgk

// ---------------------------------------------------------------------------
// Force of the fluid on the boundary faces of one tag (the cylinder's wall,
// Sec. 3.3: drag and lift): F = sum over the faces and their GL nodes of
// w_a w_b |J a^dir| (p n - tau n), n the unit outward normal of the fluid
// element (into the body), tau the viscous stress of the node's state and
// BR1 gradient.  One warp per face, a partial per face, then a sum in face
// order (deterministic); and its vector-Jacobian product.
// ---------------------------------------------------------------------------
namespace {

template <typename S>
__device__ __forceinline__ void wall_traction(const DevPhys& ph, const S q[5], const S* g, bool ns, const double nv[3],
                                              S t[3]) {
  const double gm1 = ph.gamma - 1.0;
  const S p = gm1 * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]);
  for (int i = 0; i < 3; ++i) t[i] = p * nv[i];
  if (ns) {
    S fv[3][5];
    viscous_s(ph, q, g, fv);
    for (int i = 0; i < 3; ++i)
      for (int d = 0; d < 3; ++d) t[i] -= fv[d][1 + i] * nv[d];
  }
}

template <bool AFFINE, bool NS>
__global__ void __launch_bounds__(32 * kFaceWarps) wall_force_kernel(FaceParams P, int tag, double* partial) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int fidx = blockIdx.x * kFaceWarps + warp;
  if (fidx >= P.n_faces) return;
  const FaceRec fr = P.faces[fidx];
  if (bad_face(P.m, fr)) return;
  double acc[3] = {0.0, 0.0, 0.0};
  if (fr.kind == 2 && fr.R == tag) {
    const MeshView& m = P.m;
    const int e = fr.L, f = fr.face, dir = f >> 1, side = f & 1;
    int n1, n2, n3;
    orders_of(m, e, n1, n2, n3);
    const int n = n1 * n2 * n3;
    const int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3, nf = na * nb;
    const int64_t o = m.off[e];
    const double* wa = P.basis + c_boff.W[na - 1];
    const double* wb = P.basis + c_boff.W[nb - 1];
    for (int p = lane; p < nf; p += 32) {
      const int a = p % na, b = p / na;
      const int vi = face_vidx(n1, n2, n3, f, a, b);
      double ja[3], nv[3], q[5], g[15], t[3];
      face_metric<AFFINE>(m, e, n, vi, dir, ja);
      const double area = unit_normal(ja, nv);
      for (int c = 0; c < 3; ++c) nv[c] *= side ? 1.0 : -1.0;
      for (int v = 0; v < 5; ++v) q[v] = P.q[5 * o + v * n + vi];
      if (NS)
        for (int v = 0; v < 5; ++v)
          for (int c = 0; c < 3; ++c) g[v * 3 + c] = P.grad[15 * o + (c * 5 + v) * n + vi];
      wall_traction(m.ph, q, g, NS, nv, t);
      const double wgt = __ldg(wa + a) * __ldg(wb + b) * area;
      for (int i = 0; i < 3; ++i) acc[i] += wgt * t[i];
    }
  }
  for (int i = 0; i < 3; ++i)
    for (int off = 16; off > 0; off >>= 1) acc[i] += __shfl_down_sync(0xffffffffu, acc[i], off);
  if (lane == 0)
    for (int i = 0; i < 3; ++i) partial[3 * fidx + i] = acc[i];
}

// The three components summed over the per-face partials in a fixed order
// (deterministic): each thread sums a strided subset, then a tree over the block.
constexpr int kForceSumThreads = 256;
__global__ void __launch_bounds__(kForceSumThreads) force_sum_kernel(const double* partial, int n_faces, double* F) {
  __shared__ double red[3][kForceSumThreads];
  double s[3] = {0.0, 0.0, 0.0};
  for (int f = threadIdx.x; f < n_faces; f += kForceSumThreads)
    for (int c = 0; c < 3; ++c) s[c] += partial[3 * f + c];
  for (int c = 0; c < 3; ++c) red[c][threadIdx.x] = s[c];
  __syncthreads();
  for (int h = kForceSumThreads / 2; h > 0; h >>= 1) {
    if (threadIdx.x < h)
      for (int c = 0; c < 3; ++c) red[c][threadIdx.x] += red[c][threadIdx.x + h];
    __syncthreads();
  }
  if (threadIdx.x < 3) F[threadIdx.x] = red[threadIdx.x][0];
}

// the force's cotangent lam (3, device) onto the wall nodes' traces (sadj)
// and, for Navier-Stokes, gradients (gadj)
template <bool AFFINE, bool NS>
__global__ void __launch_bounds__(32 * kFaceWarps) wall_force_vjp_kernel(FaceParams P, int tag, const double* lam,
                                                                          double* sadj, double* gadj) {
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int fidx = blockIdx.x * kFaceWarps + warp;
  if (fidx >= P.n_faces) return;
  const FaceRec fr = P.faces[fidx];
  if (bad_face(P.m, fr)) return;
  if (fr.kind != 2 || fr.R != tag) return;
  const MeshView& m = P.m;
  const int e = fr.L, f = fr.face, dir = f >> 1, side = f & 1;
  int n1, n2, n3;
  orders_of(m, e, n1, n2, n3);
  const int n = n1 * n2 * n3;
  const int na = dir == 0 ? n2 : n1, nb = dir == 2 ? n2 : n3, nf = na * nb;
  const int64_t o = m.off[e];
  const int64_t fo = m.soff[e] + face_offset(n1, n2, n3, f);
  const double* wa = P.basis + c_boff.W[na - 1];
  const double* wb = P.basis + c_boff.W[nb - 1];
  const double l0 = lam[0], l1 = lam[1], l2 = lam[2];
  for (int p = lane; p < nf; p += 32) {
    const int a = p % na, b = p / na;
    const int vi = face_vidx(n1, n2, n3, f, a, b);
    double ja[3], nv[3], q[5], g[15];
    face_metric<AFFINE>(m, e, n, vi, dir, ja);
    const double area = unit_normal(ja, nv);
    for (int c = 0; c < 3; ++c) nv[c] *= side ? 1.0 : -1.0;
    for (int v = 0; v < 5; ++v) q[v] = P.q[5 * o + v * n + vi];
    if (NS)
      for (int v = 0; v < 5; ++v)
        for (int c = 0; c < 3; ++c) g[v * 3 + c] = P.grad[15 * o + (c * 5 + v) * n + vi];
    const double wgt = __ldg(wa + a) * __ldg(wb + b) * area;
    const int nk = NS ? 20 : 5;
    for (int k = 0; k < nk; ++k) {
      Dual qd[5], gd[15], t[3];
      for (int v = 0; v < 5; ++v) qd[v] = {q[v], k == v ? 1.0 : 0.0};
      if (NS)
        for (int c = 0; c < 15; ++c) gd[c] = {g[c], k == 5 + c ? 1.0 : 0.0};
      wall_traction(m.ph, qd, gd, NS, nv, t);
      const double s = wgt * (l0 * t[0].d + l1 * t[1].d + l2 * t[2].d);
      if (k < 5) sadj[5 * fo + k * nf + p] = s;
      else gadj[15 * fo + (k - 5) * nf + p] = s;   // g index v*3+c: the gadj layout [v][c]
    }
  }
}

}  // namespace

namespace dgk {

cudaError_t wall_force(dg_mesh_impl* m, const double* q, int tag, double* F) {
  cudaError_t err;
  const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
  if (ns && ((err = face_qhat(m, q)) || (err = gradient(m, q, m->d_grad, false)))) return err;
  FaceParams P = dgk_face_params_for(m, q, nullptr);
  P.grad = m->d_grad;
  const int nfc = std::max(m->n_faces, 1);
  const int grid = (nfc + kFaceWarps - 1) / kFaceWarps;
  Prof pr(m, DG_KERNEL_ADJOINT, m->n_faces ? 2 : 1);
  if (!m->n_faces) return cudaMemsetAsync(F, 0, 3 * sizeof(double), m->stream);
  if (ns) {
    if (m->affine) wall_force_kernel<true, true><<<grid, 32 * kFaceWarps, 0, m->stream>>>(P, tag, m->d_force);
    else wall_force_kernel<false, true><<<grid, 32 * kFaceWarps, 0, m->stream>>>(P, tag, m->d_force);
  } else {
    if (m->affine) wall_force_kernel<true, false><<<grid, 32 * kFaceWarps, 0, m->stream>>>(P, tag, m->d_force);
    else wall_force_kernel<false, false><<<grid, 32 * kFaceWarps, 0, m->stream>>>(P, tag, m->d_force);
  }
  if ((err = cudaGetLastError())) return err;
  force_sum_kernel<<<1, kForceSumThreads, 0, m->stream>>>(m->d_force, m->n_faces, F);
  return cudaGetLastError();
}

// out = (dF/dq)^T lam, or out += (*scale) (dF/dq)^T lam
cudaError_t wall_force_vjp(dg_mesh_impl* m, const double* q, int tag, const double* lam, double* out,
                           const double* scale) {
  cudaError_t err;
  const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
  if (ns && ((err = face_qhat(m, q)) || (err = gradient(m, q, m->d_grad, false)))) return err;
  const size_t sf = (size_t)m->h_soff[m->n_elem];
  const int64_t ns5 = 5 * m->n_nodes;
  if ((err = cudaMemsetAsync(m->d_sadj, 0, sizeof(double) * 5 * sf, m->stream))) return err;
  if ((err = cudaMemsetAsync(m->d_adjt, 0, sizeof(double) * ns5, m->stream))) return err;
  if (ns) {
    if ((err = cudaMemsetAsync(m->d_gadj, 0, sizeof(double) * 15 * sf, m->stream))) return err;
    if ((err = cudaMemsetAsync(m->d_lG, 0, sizeof(double) * 15 * m->n_nodes, m->stream))) return err;
  }
  Prof pr(m, DG_KERNEL_ADJOINT, 1);
  if (m->n_faces) {
    FaceParams P = dgk_face_params_for(m, q, nullptr);
    P.grad = m->d_grad;
    const int grid = (m->n_faces + kFaceWarps - 1) / kFaceWarps;
    if (ns) {
      if (m->affine) wall_force_vjp_kernel<true, true><<<grid, 32 * kFaceWarps, 0, m->stream>>>(P, tag, lam, m->d_sadj, m->d_gadj);
      else wall_force_vjp_kernel<false, true><<<grid, 32 * kFaceWarps, 0, m->stream>>>(P, tag, lam, m->d_sadj, m->d_gadj);
    } else {
      if (m->affine) wall_force_vjp_kernel<true, false><<<grid, 32 * kFaceWarps, 0, m->stream>>>(P, tag, lam, m->d_sadj, nullptr);
      else wall_force_vjp_kernel<false, false><<<grid, 32 * kFaceWarps, 0, m->stream>>>(P, tag, lam, m->d_sadj, nullptr);
    }
    if ((err = cudaGetLastError())) return err;
  }
  AdjParams A;
  memset(&A, 0, sizeof(A));
  A.m = view(m);
  A.items = m->d_vitems;
  A.n_items_all = m->n_vitems;
  A.elist = m->d_velist;
  A.q = q;
  A.grad = m->d_grad;
  A.basis = m->basis64;
  A.out = m->d_adjt;
  if (ns) {   // the gradients' cotangents through BR1, then q-hat
    A.gout = m->d_lG;
    A.gadj = m->d_gadj;
    A.lS = m->d_lS;
    for (auto& c : m->vol_classes) {
      A.ilist = c.d_list;
      A.n_items = c.n;
      const size_t smem = sizeof(double) * 15 * c.S;
      if (m->affine) {
        if ((err = allow_smem(adj_gradient_kernel<true>, smem))) return err;
        adj_gradient_kernel<true><<<c.n, kVolThreads, smem, m->stream>>>(A);
      } else {
        if ((err = allow_smem(adj_gradient_kernel<false>, smem))) return err;
        adj_gradient_kernel<false><<<c.n, kVolThreads, smem, m->stream>>>(A);
      }
      if ((err = cudaGetLastError())) return err;
    }
    if ((err = adj_qhat_all(m, q, nullptr, nullptr))) return err;
  }
  A.sadj = m->d_sadj;
  for (auto& c : m->vol_classes) {
    A.ilist = c.d_list;
    A.n_items = c.n;
    adj_gather_kernel<<<c.n, kVolThreads, 0, m->stream>>>(A);
    if ((err = cudaGetLastError())) return err;
  }
  if (!scale) return cudaMemcpyAsync(out, m->d_adjt, sizeof(double) * ns5, cudaMemcpyDeviceToDevice, m->stream);
  const int grid = grid_for((int)std::min<int64_t>((ns5 + 255) / 256, 1 << 20), 8);
  axpy_dev_kernel<<<grid, 256, 0, m->stream>>>(out, m->d_adjt, scale, ns5);
  return cudaGetLastError();
}

}  // namespace dgk
