// capi.cpp -- mesh construction (host) and the extern "C" entry points of
// libdg declared in include/dg.h.
#include <algorithm>
#include <array>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <map>
#include <tuple>
#include <vector>

#include "dg_internal.h"

namespace {

// ------------------------------------------------------------ basis upload
struct DeviceBasis {
  bool ready = false;
  const double* d64 = nullptr;
  const float* d32 = nullptr;
  BasisOffsets off{};
};
DeviceBasis g_basis[64];
std::vector<double> g_tables;
BasisOffsets g_off;
bool g_tables_built = false;

void ensure_tables() {
  if (!g_tables_built) {
    dgb::build_tables(&g_off, &g_tables);
    g_tables_built = true;
  }
}

cudaError_t ensure_device_basis(int dev) {
  ensure_tables();
  if (dev < 0 || dev >= 64) return cudaErrorInvalidDevice;
  DeviceBasis& b = g_basis[dev];
  if (!b.ready) {
    dgk::upload_basis(dev, g_off, g_tables, &b.d64, &b.d32);
    cudaError_t e = cudaGetLastError();
    if (e) return e;
    b.off = g_off;
    b.ready = true;
  }
  return cudaSuccess;
}

// -------------------------------------------------------------- geometry
// Apply a (nt x nf) matrix along direction dir of a 3D array (ext[dir] == nf).
void tensor_apply(const double* A, int nt, int nf, int dir, const int ext[3], const double* in, double* out) {
  int eo[3] = {ext[0], ext[1], ext[2]};
  eo[dir] = nt;
  int stride = dir == 0 ? 1 : (dir == 1 ? ext[0] : ext[0] * ext[1]);
  for (int k = 0; k < eo[2]; ++k)
    for (int j = 0; j < eo[1]; ++j)
      for (int i = 0; i < eo[0]; ++i) {
        int r = dir == 0 ? i : (dir == 1 ? j : k);
        int ii = dir == 0 ? 0 : i, jj = dir == 1 ? 0 : j, kk = dir == 2 ? 0 : k;
        int base = ii + ext[0] * (jj + ext[1] * kk);
        double s = 0.0;
        for (int mm = 0; mm < nf; ++mm) s += A[r * nf + mm] * in[base + mm * stride];
        out[i + eo[0] * (j + eo[1] * k)] = s;
      }
}

// Node coordinates X[3][n], metric terms Ja[3][3][n] (J a^i_d) and J[n] of one
// element at orders N.  The element map is the degree-G tensor polynomial
// through the equispaced geometry lattice; J a^i in Kopriva's conservative
// curl form: J a^i_n = -e_i . curl_xi( I^N( X_l grad_xi X_m ) ), (n,m,l)
// cyclic, which makes sum_i d(J a^i)/dxi_i vanish discretely (free-stream
// preservation on curved elements).
void element_geometry(const double* gnodes, int G, const int N[3], std::vector<double>& X, std::vector<double>& Ja,
                      std::vector<double>& J) {
  const int ng = G + 1;
  const int n = (N[0] + 1) * (N[1] + 1) * (N[2] + 1);
  X.assign(3 * n, 0.0);
  Ja.assign(9 * n, 0.0);
  J.assign(n, 0.0);
  double xs[DG_NP1 + 8];
  for (int a = 0; a <= G; ++a) xs[a] = -1.0 + 2.0 * a / G;
  double E[3][DG_NP1 * 16], D[3][DG_NP1 * DG_NP1];
  for (int d = 0; d < 3; ++d) {
    double x[DG_NP1], w[DG_NP1];
    dgb::gl_nodes_weights(N[d], x, w);
    dgb::interp_matrix(xs, ng, x, N[d] + 1, E[d]);
    dgb::deriv_matrix(N[d], D[d]);
  }
  std::vector<double> a(std::max(n, ng * ng * ng) * 2), b(std::max(n, ng * ng * ng) * 2);
  for (int c = 0; c < 3; ++c) {
    for (int p = 0; p < ng * ng * ng; ++p) a[p] = gnodes[3 * p + c];
    int ext[3] = {ng, ng, ng};
    for (int d = 0; d < 3; ++d) {
      tensor_apply(E[d], N[d] + 1, ng, d, ext, a.data(), b.data());
      ext[d] = N[d] + 1;
      std::swap(a, b);
    }
    std::copy(a.begin(), a.begin() + n, X.begin() + c * n);
  }
  const int ext[3] = {N[0] + 1, N[1] + 1, N[2] + 1};
  std::vector<double> dX(9 * n);  // dX[(c*3+i)*n] = dX_c/dxi_i
  for (int c = 0; c < 3; ++c)
    for (int i = 0; i < 3; ++i) tensor_apply(D[i], N[i] + 1, N[i] + 1, i, ext, &X[c * n], &dX[(c * 3 + i) * n]);
  for (int p = 0; p < n; ++p) {
    auto g = [&](int c, int i) { return dX[(c * 3 + i) * n + p]; };
    J[p] = g(0, 0) * (g(1, 1) * g(2, 2) - g(1, 2) * g(2, 1)) - g(0, 1) * (g(1, 0) * g(2, 2) - g(1, 2) * g(2, 0)) +
           g(0, 2) * (g(1, 0) * g(2, 1) - g(1, 1) * g(2, 0));
  }
  std::vector<double> W(3 * n), dW(n);
  for (int nn = 0; nn < 3; ++nn) {
    const int mm = (nn + 1) % 3, ll = (nn + 2) % 3;
    for (int jdir = 0; jdir < 3; ++jdir)
      for (int p = 0; p < n; ++p) W[jdir * n + p] = X[ll * n + p] * dX[(mm * 3 + jdir) * n + p];
    for (int i = 0; i < 3; ++i) {
      const int i1 = (i + 1) % 3, i2 = (i + 2) % 3;
      // (curl W)_i = d_{i1} W_{i2} - d_{i2} W_{i1};  J a^i_nn = -(curl W)_i
      tensor_apply(D[i1], N[i1] + 1, N[i1] + 1, i1, ext, &W[i2 * n], dW.data());
      for (int p = 0; p < n; ++p) Ja[(i * 3 + nn) * n + p] -= dW[p];
      tensor_apply(D[i2], N[i2] + 1, N[i2] + 1, i2, ext, &W[i1 * n], dW.data());
      for (int p = 0; p < n; ++p) Ja[(i * 3 + nn) * n + p] += dW[p];
    }
  }
}

// Parallelepiped test of a G=1 element; on success the affine metrics
// (J a^i = cross products of the edge vectors / 4, J = triple product / 8).
bool affine_metrics(const double* c, double met[16]) {
  double e1[3], e2[3], e3[3], scale = 0.0;
  for (int d = 0; d < 3; ++d) {
    e1[d] = c[3 * 1 + d] - c[3 * 0 + d];
    e2[d] = c[3 * 2 + d] - c[3 * 0 + d];
    e3[d] = c[3 * 4 + d] - c[3 * 0 + d];
    scale = std::max(scale, std::fabs(e1[d]) + std::fabs(e2[d]) + std::fabs(e3[d]));
  }
  const int comb[4][4] = {{3, 1, 1, 0}, {5, 1, 0, 1}, {6, 0, 1, 1}, {7, 1, 1, 1}};
  for (auto& cb : comb)
    for (int d = 0; d < 3; ++d) {
      double expect = c[d] + cb[1] * e1[d] + cb[2] * e2[d] + cb[3] * e3[d];
      if (std::fabs(c[3 * cb[0] + d] - expect) > 1e-13 * scale) return false;
    }
  double a1[3], a2[3], a3[3];
  for (int d = 0; d < 3; ++d) { a1[d] = 0.5 * e1[d]; a2[d] = 0.5 * e2[d]; a3[d] = 0.5 * e3[d]; }
  auto cross = [](const double* x, const double* y, double* z) {
    z[0] = x[1] * y[2] - x[2] * y[1];
    z[1] = x[2] * y[0] - x[0] * y[2];
    z[2] = x[0] * y[1] - x[1] * y[0];
  };
  cross(a2, a3, met + 0);
  cross(a3, a1, met + 3);
  cross(a1, a2, met + 6);
  met[9] = a1[0] * met[0] + a1[1] * met[1] + a1[2] * met[2];
  return true;
}

template <typename T>
cudaError_t upload(T** dst, const T* src, size_t n) {
  if (n == 0) n = 1;
  cudaError_t e = cudaMalloc(dst, sizeof(T) * n);
  if (e) return e;
  if (src) return cudaMemcpy(*dst, src, sizeof(T) * n, cudaMemcpyHostToDevice);
  return cudaSuccess;
}

void free_device(dg_mesh_impl* m) {
  void* ptrs[] = {m->d_mfaces, m->d_mbatches, m->d_ord, m->d_nbr, m->d_off, m->d_soff, m->d_metric, m->d_metric32, m->d_surf, m->d_trace, m->d_surfq,
                  m->d_grad, m->d_xyz, m->d_faces, m->d_fnodes, m->d_items, m->d_elist, m->d_err, m->d_scratch,
                  m->d_taugeo,
                  m->d_taugeo32, m->d_taugeo_off, m->d_rp, m->d_rp32, m->d_qc, m->d_rc, m->d_sweep, m->d_adv,
                  m->d_vitems, m->d_velist, m->d_sadj, m->d_adjw, m->d_gadj, m->d_lG, m->d_lS, m->d_adjt,
                  m->d_force, m->d_geom, m->d_hq, m->d_hg, m->d_ht, m->d_hmap_new, m->d_hmap_trad};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  m->d_ord = nullptr; m->d_nbr = nullptr; m->d_off = nullptr; m->d_soff = nullptr; m->d_metric = nullptr;
  m->d_metric32 = nullptr; m->d_surf = nullptr; m->d_trace = nullptr; m->d_surfq = nullptr; m->d_grad = nullptr; m->d_xyz = nullptr;
  m->d_faces = nullptr; m->d_fnodes = nullptr; m->d_items = nullptr; m->d_elist = nullptr; m->d_err = nullptr; m->d_scratch = nullptr;
  m->d_taugeo = nullptr; m->d_taugeo32 = nullptr; m->d_taugeo_off = nullptr; m->d_rp = nullptr; m->d_qc = nullptr;
  m->d_rc = nullptr; m->d_sweep = nullptr; m->d_mfaces = nullptr; m->d_mbatches = nullptr; m->d_rp32 = nullptr;
  m->d_adv = nullptr;
  m->d_vitems = nullptr;
  m->d_velist = nullptr;
  m->d_sadj = nullptr;
  m->d_adjw = nullptr;
  m->d_gadj = nullptr;
  m->d_lG = nullptr;
  m->d_lS = nullptr;
  m->d_adjt = nullptr;
  m->d_force = nullptr;
  m->d_geom = nullptr;
  m->d_hq = m->d_hg = m->d_ht = nullptr;
  m->d_hmap_new = m->d_hmap_trad = nullptr;
  m->hmap_bytes = 0;
}

void destroy_impl(dg_mesh_impl* m) {
  if (!m) return;
  for (auto& c : m->tau_classes) cudaFree(c.d_list);
  m->tau_classes.clear();
  for (auto& c : m->vol_classes) cudaFree(c.d_list);
  m->vol_classes.clear();
  for (auto* u : m->tau_units) if (u) cudaFree(u);
  m->tau_units.clear();
  for (auto* u : m->tau_units_split) if (u) cudaFree(u);
  m->tau_units_split.clear();
  if (m->d_tgroups) cudaFree(m->d_tgroups);
  if (m->d_tgentries) cudaFree(m->d_tgentries);
  m->d_tgroups = m->d_tgentries = nullptr;
  for (auto& pp : m->prof_pending) {
    cudaEventDestroy(pp.a);
    cudaEventDestroy(pp.b);
  }
  for (auto ev : m->prof_pool) cudaEventDestroy(ev);
  if (m->prof_open) cudaEventDestroy(m->prof_open);
  for (auto* c : m->coarse) destroy_impl(c);
  m->coarse.clear();
  dg_advance_release(m);
  free_device(m);
  delete static_cast<dg_mesh*>(m);
}

#define DG_CUDA(x)                   \
  do {                               \
    cudaError_t _e = (x);            \
    if (_e != cudaSuccess) {         \
      return _e == cudaErrorMemoryAllocation ? DG_ERR_NOMEM : DG_ERR_CUDA; \
    }                                \
  } while (0)

constexpr int kTileNodes = 256;
constexpr size_t kGeneralMortarBytes = 96 * 1024;
constexpr int kMinTauUnits = 8 * 152;   // tau units of a size class below which groups are not shared

}  // namespace

// Mortar batches from the shape groups: per group, batches of at most the
// budget of its mortar-size class in mortar nodes (one face at least),
// largest batches first (the kernel runs one CTA per batch, and the block
// scheduler then fills the tail with the small ones).  Uploads the face list
// and the batch records.
dg_status build_mortar_batches(dg_mesh_impl* m) {
  std::vector<int32_t> mfaces, mbatches;
  m->mortar_smem = 0;
  const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
  for (const auto& g : m->h_mgroups) {
    const int nm = std::max(g.la, g.ra) * std::max(g.lb, g.rb);
    int per = std::max(1, m->mortar_budget[mortar_size_class(nm)] / nm);
    if (m->general_mortars) {   // at most 96 KB of shared memory per batch: two CTAs per SM
      const size_t one = dg_mortar_general_smem_doubles(1, g.la, g.lb, g.ra, g.rb, ns);
      per = std::max(1, std::min(per, (int)(kGeneralMortarBytes / (sizeof(double) * one))));
    }
    const int nf = (int)g.faces.size() / 3;
    for (int i = 0; i < nf; i += per) {
      const int cnt = std::min(per, nf - i);
      mbatches.insert(mbatches.end(), {(int32_t)(mfaces.size() / 3), cnt, g.la, g.lb, g.ra, g.rb});
      mfaces.insert(mfaces.end(), g.faces.begin() + 3 * i, g.faces.begin() + 3 * (i + cnt));
      m->mortar_smem = std::max(m->mortar_smem, m->general_mortars
                                                    ? dg_mortar_general_smem_doubles(cnt, g.la, g.lb, g.ra, g.rb, ns)
                                                    : dg_mortar_smem_doubles(cnt, g.la, g.lb, g.ra, g.rb));
    }
  }
  m->n_mbatches = (int)mbatches.size() / 6;
  auto cost = [&](int b) {
    const int32_t* B = &mbatches[6 * b];
    const long la = B[2], lb = B[3], ra = B[4], rb = B[5];
    const long Ma = std::max(la, ra), Mb = std::max(lb, rb);
    long c = Ma * Mb * 165;
    for (int s = 0; s < 2; ++s) {
      const long a = s ? ra : la, bb = s ? rb : lb;
      c += 20 * a * Ma * bb * (a != Ma) + 20 * bb * Ma * Mb * (bb != Mb);
    }
    return c * B[1];
  };
  std::vector<int> order(m->n_mbatches);
  for (int b = 0; b < m->n_mbatches; ++b) order[b] = b;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) { return cost(a) > cost(b); });
  m->h_mbatches.assign(mbatches.size(), 0);
  for (int b = 0; b < m->n_mbatches; ++b)
    std::copy(mbatches.begin() + 6 * order[b], mbatches.begin() + 6 * order[b] + 6, m->h_mbatches.begin() + 6 * b);
  if (m->d_mfaces) cudaFree(m->d_mfaces);
  if (m->d_mbatches) cudaFree(m->d_mbatches);
  m->d_mfaces = nullptr;
  m->d_mbatches = nullptr;
  m->n_mfaces = (int)mfaces.size() / 3;
  DG_CUDA(upload(&m->d_mfaces, mfaces.data(), mfaces.size()));
  DG_CUDA(upload(&m->d_mbatches, m->h_mbatches.data(), m->h_mbatches.size()));
  return DG_OK;
}

// Volume tiles from the order buckets: per bucket, tiles of at most the budget
// of its element-size class in nodes (one element at least).
dg_status build_volume_items(dg_mesh_impl* m) {
  std::vector<WorkItem> items;
  std::vector<int32_t> elist;
  for (size_t b = 0; b < m->h_buckets.size(); ++b) {
    const int n1 = m->h_bucket_key[b][0], n2 = m->h_bucket_key[b][1], n3 = m->h_bucket_key[b][2];
    const int n = (n1 + 1) * (n2 + 1) * (n3 + 1);
    const int per = std::max(1, m->vol_budget[elem_size_class(n)] / n);
    const auto& els = m->h_buckets[b];
    for (size_t i = 0; i < els.size(); i += per) {
      const int cnt = (int)std::min<size_t>(per, els.size() - i);
      items.push_back({(int32_t)elist.size(), cnt, n1, n2, n3});
      for (int c = 0; c < cnt; ++c) elist.push_back(els[i + c]);
    }
  }
  m->n_vitems = (int)items.size();
  m->h_vitems = items;
  // three launches by tile size, each with shared memory for its largest
  // tile (20 doubles a node): up to 400 nodes (<= 64 KB, three CTAs per SM),
  // up to 700 (<= 112 KB, two CTAs per SM) and larger ones (one CTA per SM), so
  // that a few 9^3 elements do not set the occupancy of all the others; in
  // each, the largest tiles first
  std::vector<std::vector<int32_t>> cl(3);
  std::vector<int> cS(3, 0);
  for (int i = 0; i < (int)items.size(); ++i) {
    const WorkItem& w = items[i];
    const int tile = w.count * (w.n1 + 1) * (w.n2 + 1) * (w.n3 + 1);
    const int k = tile <= 400 ? 0 : (tile <= 700 ? 1 : 2);
    cl[k].push_back(i);
    cS[k] = std::max(cS[k], tile);
  }
  auto vcost = [&](int i) {
    const WorkItem& w = items[i];
    const long n = (long)(w.n1 + 1) * (w.n2 + 1) * (w.n3 + 1);
    return w.count * n * (134 + 10 * (w.n1 + w.n2 + w.n3 + 3));
  };
  for (auto& v : cl) std::stable_sort(v.begin(), v.end(), [&](int a, int b) { return vcost(a) > vcost(b); });
  for (auto& c : m->vol_classes) cudaFree(c.d_list);
  m->vol_classes.clear();
  if (m->d_vitems) cudaFree(m->d_vitems);
  if (m->d_velist) cudaFree(m->d_velist);
  m->d_vitems = nullptr;
  m->d_velist = nullptr;
  DG_CUDA(upload(&m->d_vitems, items.data(), items.size()));
  DG_CUDA(upload(&m->d_velist, elist.data(), elist.size()));
  for (int k = 0; k < 3; ++k) {
    if (cl[k].empty()) continue;
    dg_mesh_impl::TauClass c{nullptr, (int)cl[k].size(), cS[k]};
    DG_CUDA(upload(&c.d_list, cl[k].data(), cl[k].size()));
    m->vol_classes.push_back(c);
  }
  return DG_OK;
}

namespace {

// Build every host and device structure of a mesh from its host arrays.
dg_status build(dg_mesh_impl* m) {
  const int ne = m->n_elem;
  const int G = m->G;
  const int ng3 = (G + 1) * (G + 1) * (G + 1);
  m->max_order = 1;
  for (int e = 0; e < ne; ++e) {
    const int* N = &m->h_ord[3 * e];
    for (int d = 0; d < 3; ++d) {
      if (N[d] < 1 || N[d] > DG_MAX_ORDER) return DG_ERR_ARG;
      m->max_order = std::max(m->max_order, N[d]);
    }
  }
  // geometry
  // metric record: fields 0..8 J a^i_d, 9 J, 10 1/J; affine: 16 doubles per
  // element with 11..13 |J a^i|, curved: [11][n] per element
  std::vector<double> met;
  m->affine = (G == 1);
  if (m->affine) {
    met.assign(16 * (size_t)ne, 0.0);
    for (int e = 0; e < ne && m->affine; ++e)
      if (!affine_metrics(&m->h_geom[(size_t)e * ng3 * 3], &met[16 * (size_t)e])) m->affine = false;
  }
  m->axis = m->affine;
  if (m->affine) {
    for (int e = 0; e < ne; ++e) {
      double* r = &met[16 * (size_t)e];
      if (!(r[9] > 0.0)) return DG_ERR_ARG;
      r[10] = 1.0 / r[9];
      for (int i = 0; i < 3; ++i)
        r[11 + i] = std::sqrt(r[3 * i] * r[3 * i] + r[3 * i + 1] * r[3 * i + 1] + r[3 * i + 2] * r[3 * i + 2]);
      for (int i = 0; i < 3; ++i)
        for (int d = 0; d < 3; ++d)
          if (i != d && r[3 * i + d] != 0.0) m->axis = false;
    }
  }
  const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
  // offsets; on the device build also the warp-list faces and the sorted
  // buckets and batched faces (dg_device_lists)
  DgDeviceLists dl;
  if (m->device_build) {
    DG_CUDA(upload(&m->d_ord, m->h_ord.data(), m->h_ord.size()));
    DG_CUDA(upload(&m->d_nbr, m->h_nbr.data(), m->h_nbr.size()));
    dg_status st = dg_device_lists(m, !ns && m->affine, &dl);
    if (st != DG_OK) return st;
    m->h_off.swap(dl.off);
    m->h_soff.swap(dl.soff);
  } else {
    m->h_off.assign(ne + 1, 0);
    m->h_soff.assign(ne + 1, 0);
    for (int e = 0; e < ne; ++e) {
      const int* N = &m->h_ord[3 * e];
      int64_t a = N[0] + 1, b = N[1] + 1, c = N[2] + 1;
      m->h_off[e + 1] = m->h_off[e] + a * b * c;
      m->h_soff[e + 1] = m->h_soff[e] + 2 * (b * c + a * c + a * b);
    }
  }
  m->n_nodes = m->h_off[ne];
  if (!m->affine && m->device_build) {
    // curved metrics at the element orders on the device
    if (!m->d_geom) DG_CUDA(upload(&m->d_geom, m->h_geom.data(), m->h_geom.size()));
    DG_CUDA(upload<double>(&m->d_metric, nullptr, 11 * (size_t)m->n_nodes));
    std::vector<DgGeomJob> jobs(ne);
    for (int e = 0; e < ne; ++e)
      jobs[e] = {e, m->h_ord[3 * e] + 1, m->h_ord[3 * e + 1] + 1, m->h_ord[3 * e + 2] + 1, 11 * m->h_off[e]};
    dg_status st = dg_device_metrics(m, jobs, 11, m->d_metric, nullptr);
    if (st != DG_OK) return st;
  } else if (!m->affine) {
    met.assign(11 * (size_t)m->n_nodes, 0.0);
    int bad_jacobian = 0;
#pragma omp parallel for schedule(dynamic, 8) reduction(| : bad_jacobian)
    for (int e = 0; e < ne; ++e) {
      std::vector<double> X, Ja, J;
      element_geometry(&m->h_geom[(size_t)e * ng3 * 3], G, &m->h_ord[3 * e], X, Ja, J);
      const int64_t n = m->h_off[e + 1] - m->h_off[e];
      double* dst = &met[11 * m->h_off[e]];
      for (int k = 0; k < 9; ++k) std::copy(Ja.begin() + k * n, Ja.begin() + (k + 1) * n, dst + k * n);
      for (int64_t p = 0; p < n; ++p) {
        if (!(J[p] > 0.0)) bad_jacobian = 1;
        dst[9 * n + p] = J[p];
        dst[10 * n + p] = 1.0 / J[p];
      }
    }
    if (bad_jacobian) return DG_ERR_ARG;
  }
  // faces
  std::vector<FaceRec> faces;
  std::vector<int32_t> fnodes;
  std::map<std::tuple<int, int, int, int>, std::vector<int32_t>> msig;
  const bool batch_conforming = !ns && m->affine;
  if (m->device_build) {
    m->n_face_conf = dl.n_conf;
    m->n_face_mortar = dl.n_mortar;
    m->n_face_bnd = dl.n_bnd;
    for (size_t i = 0; i < dl.msig.size(); ++i) {
      const int sg = dl.msig[i];
      auto& v = msig[std::make_tuple(sg >> 12, (sg >> 8) & 15, (sg >> 4) & 15, sg & 15)];
      v.insert(v.end(), dl.mfaces.begin() + 3 * i, dl.mfaces.begin() + 3 * i + 3);
    }
  } else {
  for (int e = 0; e < ne; ++e)
    for (int d = 0; d < 3; ++d) {
      const int t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
      for (int side = 0; side < 2; ++side) {
        const int f = 2 * d + side;
        const int nb = m->h_nbr[6 * e + f];
        if (nb >= 0) {
          if (nb >= ne || m->h_nbr[6 * nb + (f ^ 1)] != e) return DG_ERR_ARG;
          if (side == 1) {
            bool conf = m->h_ord[3 * e + t0] == m->h_ord[3 * nb + t0] && m->h_ord[3 * e + t1] == m->h_ord[3 * nb + t1];
            faces.push_back({e, nb, d, conf ? 0 : 1});
          }
        } else {
          if (nb != DG_BC_FARFIELD && nb != DG_BC_WALL) return DG_ERR_ARG;
          faces.push_back({e, nb, f, 2});
        }
      }
    }
  std::stable_sort(faces.begin(), faces.end(), [](const FaceRec& a, const FaceRec& b) { return a.kind < b.kind; });
  m->n_face_conf = m->n_face_mortar = m->n_face_bnd = 0;
  for (auto& f : faces) (f.kind == 0 ? m->n_face_conf : f.kind == 1 ? m->n_face_mortar : m->n_face_bnd)++;
  // p-nonconforming faces leave the warp-per-face list: batched by shape.  On
  // affine Euler meshes the conforming interior faces join them: the batched
  // kernel keeps every lane busy, while one warp per face leaves lanes idle
  // whenever a face has not a multiple of 32 nodes.
  std::vector<FaceRec> wfaces;
  for (auto& f : faces) {
    if (!(f.kind == 1 || (f.kind == 0 && batch_conforming))) {
      wfaces.push_back(f);
      continue;
    }
    const int d = f.face, t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
    auto key = std::make_tuple(m->h_ord[3 * f.L + t0] + 1, m->h_ord[3 * f.L + t1] + 1, m->h_ord[3 * f.R + t0] + 1,
                               m->h_ord[3 * f.R + t1] + 1);
    auto& v = msig[key];
    v.push_back(f.L);
    v.push_back(f.R);
    v.push_back(d);
  }
  faces.swap(wfaces);
  m->n_faces = (int)faces.size();
  // (face, node) of every node of the listed faces: the face kernel runs one
  // thread per face node
  for (int i = 0; i < m->n_faces; ++i) {
    const FaceRec& f = faces[i];
    const int e = f.L, d = f.kind == 2 ? f.face / 2 : f.face, t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
    const int nf = (m->h_ord[3 * e + t0] + 1) * (m->h_ord[3 * e + t1] + 1);
    for (int p = 0; p < nf; ++p) {
      fnodes.push_back(i);
      fnodes.push_back(p);
    }
  }
  m->n_fnodes = (int)fnodes.size() / 2;
  }   // host face lists
  // the batched faces by shape, faces of one direction together: the
  // axis-aligned Roe flux branches on the direction, so a warp that spans
  // two directions runs both variants
  m->h_mgroups.clear();
  for (auto& kv : msig) {
    dg_mesh_impl::MGroup g;
    std::tie(g.la, g.lb, g.ra, g.rb) = kv.first;
    const int nf = (int)kv.second.size() / 3;
    std::vector<std::array<int32_t, 3>> fs(nf);
    for (int i = 0; i < nf; ++i) fs[i] = {kv.second[3 * i], kv.second[3 * i + 1], kv.second[3 * i + 2]};
    if (!m->device_build)   // the device sort already ordered them by direction
      std::stable_sort(fs.begin(), fs.end(), [](const std::array<int32_t, 3>& a, const std::array<int32_t, 3>& b) {
        return a[2] < b[2];
      });
    g.faces.resize(3 * (size_t)nf);
    for (int i = 0; i < nf; ++i)
      for (int k = 0; k < 3; ++k) g.faces[3 * i + k] = fs[i][k];
    m->h_mgroups.push_back(std::move(g));
  }
  // mortars of curved or Navier-Stokes meshes take the general kernels (each
  // side's flux with its own normal; BR1 gradients on the mortar)
  m->general_mortars = m->n_face_mortar > 0 && (ns || !m->affine);
  {
    dg_status st = build_mortar_batches(m);
    if (st != DG_OK) return st;
  }
  // a mortar batch above the device's shared memory (one face of the largest
  // shape always fits below DG_MAX_ORDER) would refuse face-coupled calls
  {
    int dev = 0, limit = 0;
    DG_CUDA(cudaGetDevice(&dev));
    DG_CUDA(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
    m->faces_unsupported = sizeof(double) * m->mortar_smem + 1024 > (size_t)limit;
  }
  // work items: elements bucketed by order triple
  std::map<std::tuple<int, int, int>, std::vector<int32_t>> buckets;
  if (m->device_build) {   // sorted on the device: runs of equal keys
    for (int i = 0; i < ne; ++i) {
      const int k = dl.bucket_key[i];
      buckets[{k / 64 + 1, (k / 8) % 8 + 1, k % 8 + 1}].push_back(dl.bucket_elems[i]);
    }
  } else {
    for (int e = 0; e < ne; ++e) buckets[{m->h_ord[3 * e], m->h_ord[3 * e + 1], m->h_ord[3 * e + 2]}].push_back(e);
  }
  m->h_bucket_key.clear();
  m->h_buckets.clear();
  for (auto& kv : buckets) {
    m->h_bucket_key.push_back({std::get<0>(kv.first), std::get<1>(kv.first), std::get<2>(kv.first)});
    m->h_buckets.push_back(kv.second);
  }
  std::vector<WorkItem> items;
  std::vector<int32_t> elist;
  for (auto& kv : buckets) {
    int n1, n2, n3;
    std::tie(n1, n2, n3) = kv.first;
    int n = (n1 + 1) * (n2 + 1) * (n3 + 1);
    int per = std::max(1, kTileNodes / n);
    const auto& els = kv.second;
    for (size_t i = 0; i < els.size(); i += per) {
      int cnt = (int)std::min<size_t>(per, els.size() - i);
      items.push_back({(int32_t)elist.size(), cnt, n1, n2, n3});
      for (int c = 0; c < cnt; ++c) elist.push_back(els[i + c]);
    }
  }
  m->n_items = (int)items.size();
  m->h_items = items;
  // device
  if (!m->device_build) {
    DG_CUDA(upload(&m->d_ord, m->h_ord.data(), m->h_ord.size()));
    DG_CUDA(upload(&m->d_nbr, m->h_nbr.data(), m->h_nbr.size()));
    DG_CUDA(upload(&m->d_off, m->h_off.data(), m->h_off.size()));
    DG_CUDA(upload(&m->d_soff, m->h_soff.data(), m->h_soff.size()));
    DG_CUDA(upload(&m->d_faces, faces.data(), faces.size()));
    DG_CUDA(upload(&m->d_fnodes, fnodes.data(), fnodes.size()));
  }
  if (!m->device_build || m->affine) DG_CUDA(upload(&m->d_metric, met.data(), met.size()));
  if (m->affine) {
    std::vector<float> m32(met.begin(), met.end());
    DG_CUDA(upload(&m->d_metric32, m32.data(), m32.size()));
  }
  DG_CUDA(upload(&m->d_items, items.data(), items.size()));
  DG_CUDA(upload(&m->d_elist, elist.data(), elist.size()));
  DG_CUDA(upload<double>(&m->d_surf, nullptr, 5 * (size_t)m->h_soff[ne]));
  if (m->affine && !ns && m->n_mbatches)   // the mortar kernel's face traces (dgk::face_flux_rk)
    DG_CUDA(upload<double>(&m->d_trace, nullptr, 5 * (size_t)m->h_soff[ne]));
  if (ns) {
    DG_CUDA(upload<double>(&m->d_surfq, nullptr, 15 * (size_t)m->h_soff[ne]));
    DG_CUDA(upload<double>(&m->d_grad, nullptr, 15 * (size_t)m->n_nodes));
  }
  // isolated tau: the work items grouped by tile size (count * n_P) into
  // shared-memory size classes
  {
    const int bounds[5] = {64, 128, 256, 512, 1000};
    std::vector<std::vector<int32_t>> cls(5);
    std::vector<int> cS(5, 0);
    for (int i = 0; i < (int)items.size(); ++i) {
      const WorkItem& w = items[i];
      const int tile = w.count * (w.n1 + 1) * (w.n2 + 1) * (w.n3 + 1);
      int k = 0;
      while (tile > bounds[k]) ++k;
      cls[k].push_back(i);
      cS[k] = std::max(cS[k], tile);
    }
    for (int k = 0; k < 5; ++k) {
      if (cls[k].empty()) continue;
      dg_mesh_impl::TauClass c{nullptr, (int)cls[k].size(), cS[k]};
      DG_CUDA(upload(&c.d_list, cls[k].data(), cls[k].size()));
      m->tau_classes.push_back(c);
    }
  }
  {
    dg_status st = build_volume_items(m);
    if (st != DG_OK) return st;
  }
  DG_CUDA(upload<unsigned>(&m->d_err, nullptr, 1));
  DG_CUDA(cudaMemset(m->d_err, 0, sizeof(unsigned)));
  DG_CUDA(upload<double>(&m->d_scratch, nullptr, 4));
  DG_CUDA(cudaGetDevice(&m->device));
  DG_CUDA(ensure_device_basis(m->device));
  m->basis64 = g_basis[m->device].d64;
  m->basis32 = g_basis[m->device].d32;
  m->boff = g_basis[m->device].off;
  return DG_OK;
}

// Metrics at every coarse order N <= P of every element (curved meshes, for
// the isolated tau sweep): per element the combos N1 fastest, then N2, N3,
// each [10][n_N].
dg_status build_tau_bank(dg_mesh_impl* m) {
  if (m->affine || m->d_taugeo) return DG_OK;
  const int ne = m->n_elem;
  std::vector<int64_t> off(ne + 1, 0);
  std::vector<DgGeomJob> jobs;
  for (int e = 0; e < ne; ++e) {
    const int* P = &m->h_ord[3 * e];
    int64_t pos = off[e];
    for (int N3 = 1; N3 <= P[2]; ++N3)
      for (int N2 = 1; N2 <= P[1]; ++N2)
        for (int N1 = 1; N1 <= P[0]; ++N1) {
          jobs.push_back({e, N1 + 1, N2 + 1, N3 + 1, pos});
          pos += 10 * (int64_t)(N1 + 1) * (N2 + 1) * (N3 + 1);
        }
    off[e + 1] = pos;
  }
  // every (element, coarse order) on the device, one CTA each (on the host
  // cores this construction was the bulk of the first sweep on a curved mesh)
  if (!m->d_geom) DG_CUDA(upload(&m->d_geom, m->h_geom.data(), m->h_geom.size()));
  DG_CUDA(upload<double>(&m->d_taugeo, nullptr, off[ne]));
  DG_CUDA(upload<float>(&m->d_taugeo32, nullptr, off[ne]));
  dg_status st = dg_device_metrics(m, jobs, 10, m->d_taugeo, m->d_taugeo32);
  if (st != DG_OK) return st;
  DG_CUDA(upload(&m->d_taugeo_off, off.data(), off.size()));
  return DG_OK;
}

// Work units of the isolated sweep for the current sweep list: the entries
// grouped by (N2, N3), and per shared-memory class the (item, group) pairs
// whose group reaches at least one entry within the item's orders.
dg_status build_tau_units(dg_mesh_impl* m) {
  // sweep entries grouped by (N2, N3), the groups ordered by N3 then N2: a
  // unit is a tile and the groups of one N3 (the xi3 restriction is shared)
  std::map<std::pair<int, int>, std::vector<int32_t>> grp;   // key (N3, N2)
  const int ns = (int)m->h_sweep.size() / 3;
  for (int s = 0; s < ns; ++s) {
    auto& v = grp[{m->h_sweep[3 * s + 2], m->h_sweep[3 * s + 1]}];
    v.push_back(s);
    v.push_back(m->h_sweep[3 * s]);
  }
  std::vector<int32_t> groups, gentries;
  std::vector<int> gmin1;    // smallest N1 of each group
  for (auto& kv : grp) {
    int mn = 1 << 30;
    for (size_t i = 1; i < kv.second.size(); i += 2) mn = std::min(mn, kv.second[i]);
    groups.insert(groups.end(), {kv.first.second, kv.first.first, (int32_t)(gentries.size() / 2),
                                 (int32_t)(kv.second.size() / 2)});
    gentries.insert(gentries.end(), kv.second.begin(), kv.second.end());
    gmin1.push_back(mn);
  }
  for (auto* u : m->tau_units) if (u) cudaFree(u);
  for (auto* u : m->tau_units_split) if (u) cudaFree(u);
  m->tau_units.assign(m->tau_classes.size(), nullptr);
  m->tau_units_split.assign(m->tau_classes.size(), nullptr);
  m->tau_n_units.assign(m->tau_classes.size(), 0);
  m->tau_n_units_split.assign(m->tau_classes.size(), 0);
  m->tau_n_shared.assign(m->tau_classes.size(), 0);
  m->tau_last_units.clear();
  m->tau_last_shared.clear();
  if (m->d_tgroups) cudaFree(m->d_tgroups);
  if (m->d_tgentries) cudaFree(m->d_tgentries);
  m->d_tgroups = m->d_tgentries = nullptr;
  m->n_tgroups = (int)groups.size() / 4;
  m->n_tgentries = (int)gentries.size() / 2;
  DG_CUDA(upload(&m->d_tgroups, groups.data(), groups.size()));
  DG_CUDA(upload(&m->d_tgentries, gentries.data(), gentries.size()));
  for (size_t k = 0; k < m->tau_classes.size(); ++k) {
    std::vector<int32_t> ilist(m->tau_classes[k].n);
    DG_CUDA(cudaMemcpy(ilist.data(), m->tau_classes[k].d_list, sizeof(int32_t) * ilist.size(), cudaMemcpyDeviceToHost));
    std::vector<int32_t> units;   // (item, first group, group count, 0)
    const int ng = (int)groups.size() / 4;
    for (int it : ilist) {
      const WorkItem& w = m->h_items[it];
      for (int g = 0; g < ng;) {
        const int N3 = groups[4 * g + 1];
        int h = g;
        while (h < ng && groups[4 * h + 1] == N3) ++h;      // [g, h): the groups of this N3, N2 ascending
        int last = g;                                        // the prefix with N2 <= P2
        while (last < h && groups[4 * last] <= w.n2) ++last;
        bool any = false;
        for (int x = g; x < last; ++x) any = any || gmin1[x] <= w.n1;
        if (N3 <= w.n3 && last > g && any) units.insert(units.end(), {it, g, last - g, 0});
        g = h;
      }
    }
    // a small mesh keeps one group per unit: the shared xi3 restriction saves
    // work, but too few units leave SMs idle (DG_TAU_UNITS_AUTO); the other
    // modes force one form
    std::vector<int32_t> split;   // one group per unit (also what the compact FP64 layout runs)
    for (size_t u = 0; u < units.size(); u += 4)
      for (int x = units[u + 1]; x < units[u + 1] + units[u + 2]; ++x)
        if (gmin1[x] <= m->h_items[units[u]].n1) split.insert(split.end(), {units[u], x, 1, 0});
    const bool use_split = m->tau_unit_mode == DG_TAU_UNITS_SPLIT ||
                           (m->tau_unit_mode == DG_TAU_UNITS_AUTO && (int)units.size() / 4 < kMinTauUnits);
    if (use_split) units = split;
    m->tau_n_units[k] = (int)units.size() / 4;
    for (size_t u = 0; u < units.size(); u += 4) m->tau_n_shared[k] += units[u + 2] > 1;
    m->tau_n_units_split[k] = (int)split.size() / 4;
    DG_CUDA(upload(&m->tau_units[k], units.data(), units.size()));
    DG_CUDA(upload(&m->tau_units_split[k], split.data(), split.size()));
  }
  return DG_OK;
}

dg_status from_cuda(cudaError_t e) {
  if (e == cudaSuccess) return DG_OK;
  return e == cudaErrorMemoryAllocation ? DG_ERR_NOMEM : DG_ERR_CUDA;
}

dg_status residual_impl(dg_mesh_impl* m, const double* q, double* r, bool isolated) {
  if (!isolated && m->faces_unsupported) return DG_ERR_UNSUPPORTED;
  cudaError_t e;
  const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
  if (ns) {
    if (!isolated && (e = dgk::face_qhat(m, q))) return from_cuda(e);
    if ((e = dgk::gradient(m, q, m->d_grad, isolated))) return from_cuda(e);
  }
  if (!isolated && (e = dgk::face_flux(m, q, m->d_grad, false))) return from_cuda(e);
  return from_cuda(dgk::volume(m, q, m->d_grad, r, isolated, -1, nullptr, nullptr, nullptr));
}

dg_mesh_impl* make_child(const dg_mesh_impl* m, const std::vector<int32_t>& orders, dg_status* st,
                         bool on_device = false) {
  dg_mesh* c = new dg_mesh();
  c->stream = m->stream;
  c->device_build = on_device;
  c->n_elem = m->n_elem;
  c->G = m->G;
  c->phys = m->phys;
  c->h_geom = m->h_geom;
  c->h_nbr = m->h_nbr;
  c->h_ord = orders;
  std::copy(m->vol_budget, m->vol_budget + kSizeClasses, c->vol_budget);   // tuned budgets carry over
  std::copy(m->mortar_budget, m->mortar_budget + kSizeClasses, c->mortar_budget);
  *st = build(c);
  if (*st != DG_OK) {
    destroy_impl(c);
    return nullptr;
  }
  return c;
}

cudaEvent_t pool_event(dg_mesh_impl* m) {
  if (!m->prof_pool.empty()) {
    cudaEvent_t e = m->prof_pool.back();
    m->prof_pool.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

}  // namespace

// Launch hooks: count every launch; with profiling on, bracket it with a
// pair of events on the mesh stream (read back in dg_profile_read).
void dg_prof_begin(dg_mesh_impl* m, int kernel_id, int n_launches) {
  (void)kernel_id;
  m->launches += n_launches;
  if (!m->prof_on) return;
  m->prof_open = pool_event(m);
  cudaEventRecord(m->prof_open, m->stream);
}

void dg_prof_end(dg_mesh_impl* m, int kernel_id) {
  if (!m->prof_on || !m->prof_open) return;
  cudaEvent_t b = pool_event(m);
  cudaEventRecord(b, m->stream);
  m->prof_pending.push_back({kernel_id, m->prof_open, b});
  m->prof_open = nullptr;
}

// One Williamson RK3 step.  trace_valid: m->d_trace holds the face traces of
// q (the last stage of the step before wrote them and q has not changed
// since); the stages after the first always find them there.
dg_status rk_step_impl(dg_mesh_impl* m, double* q, double* g, const double* dt_dev, bool trace_valid) {
  const bool ns = m->phys.eqs == DG_NAVIER_STOKES;
  cudaError_t e;
  for (int k = 0; k < 3; ++k) {
    if (ns) {
      if ((e = dgk::face_qhat(m, q))) return from_cuda(e);
      if ((e = dgk::gradient(m, q, m->d_grad, false))) return from_cuda(e);
    }
    if ((e = dgk::face_flux_rk(m, q, k > 0 || trace_valid))) return from_cuda(e);
    if ((e = dgk::volume(m, q, m->d_grad, nullptr, false, k, q, g, dt_dev))) return from_cuda(e);
  }
  return DG_OK;
}

extern "C" {

dg_status dg_profile_enable(dg_mesh* m, int on) {
  if (!m) return DG_ERR_ARG;
  m->prof_on = on != 0;
  if (on) {
    for (int k = 0; k < DG_KERNEL_KINDS; ++k) {
      m->prof_ms[k] = 0.0;
      m->prof_n[k] = 0;
    }
  }
  return DG_OK;
}

dg_status dg_profile_read(dg_mesh* m, int kernel, double* total_ms, int64_t* launches) {
  if (!m || kernel < 0 || kernel >= DG_KERNEL_KINDS) return DG_ERR_ARG;
  DG_CUDA(m->stream ? cudaStreamSynchronize(m->stream) : cudaDeviceSynchronize());
  for (auto& pp : m->prof_pending) {
    float ms = 0.f;
    DG_CUDA(cudaEventElapsedTime(&ms, pp.a, pp.b));
    m->prof_ms[pp.id] += ms;
    m->prof_n[pp.id] += 1;
    m->prof_pool.push_back(pp.a);
    m->prof_pool.push_back(pp.b);
  }
  m->prof_pending.clear();
  if (total_ms) *total_ms = m->prof_ms[kernel];
  if (launches) *launches = m->prof_n[kernel];
  return DG_OK;
}

dg_status dg_launch_count(const dg_mesh* m, int64_t* launches) {
  if (!m || !launches) return DG_ERR_ARG;
  *launches = m->launches;
  return DG_OK;
}


const char* dg_status_str(dg_status s) {
  switch (s) {
    case DG_OK: return "ok";
    case DG_ERR_ARG: return "invalid argument";
    case DG_ERR_NOMEM: return "out of memory";
    case DG_ERR_CUDA: return "CUDA runtime error";
    case DG_ERR_UNSUPPORTED: return "unsupported configuration";
    case DG_ERR_NONPHYSICAL: return "non-physical state (rho <= 0, p <= 0 or NaN)";
    case DG_ERR_TIMEOUT: return "device wait timed out";
    case DG_ERR_INDEX: return "index out of range in a work list (bounds-checking build)";
  }
  return "unknown status";
}

dg_status dg_count_nodes(int32_t n_elem, const int32_t* orders, int64_t* n_nodes) {
  if (n_elem < 0 || (n_elem > 0 && !orders) || !n_nodes) return DG_ERR_ARG;
  int64_t s = 0;
  for (int e = 0; e < n_elem; ++e) {
    for (int d = 0; d < 3; ++d)
      if (orders[3 * e + d] < 1 || orders[3 * e + d] > DG_MAX_ORDER) return DG_ERR_ARG;
    s += (int64_t)(orders[3 * e] + 1) * (orders[3 * e + 1] + 1) * (orders[3 * e + 2] + 1);
  }
  *n_nodes = s;
  return DG_OK;
}

dg_status dg_mesh_create(const dg_mesh_desc* d, void* stream, dg_mesh** out) {
  if (!d || !out || d->n_elem <= 0 || d->geom_order < 1 || d->geom_order > 8 || !d->geom || !d->neighbors ||
      !d->orders)
    return DG_ERR_ARG;
  if (d->phys.eqs != DG_EULER && d->phys.eqs != DG_NAVIER_STOKES) return DG_ERR_ARG;
  if (!(d->phys.gamma > 1.0) || !(d->phys.Rgas > 0.0)) return DG_ERR_ARG;
  if (d->phys.eqs == DG_NAVIER_STOKES && (!(d->phys.mu >= 0.0) || !(d->phys.Pr > 0.0))) return DG_ERR_ARG;
  *out = nullptr;
  dg_mesh* m = new dg_mesh();
  m->stream = static_cast<cudaStream_t>(stream);
  m->n_elem = d->n_elem;
  m->G = d->geom_order;
  m->phys.eqs = d->phys.eqs;
  m->phys.gamma = d->phys.gamma;
  m->phys.mu = d->phys.mu;
  m->phys.Pr = d->phys.Pr;
  m->phys.Rgas = d->phys.Rgas;
  m->phys.kappa = d->phys.eqs == DG_NAVIER_STOKES
                      ? d->phys.mu * d->phys.gamma * d->phys.Rgas / ((d->phys.gamma - 1.0) * d->phys.Pr)
                      : 0.0;
  m->phys.kappa_R = d->phys.eqs == DG_NAVIER_STOKES
                        ? d->phys.mu * d->phys.gamma / ((d->phys.gamma - 1.0) * d->phys.Pr)
                        : 0.0;
  for (int v = 0; v < 5; ++v) m->phys.qinf[v] = d->phys.q_inf[v];
  const size_t ng3 = (size_t)(d->geom_order + 1) * (d->geom_order + 1) * (d->geom_order + 1);
  m->h_geom.assign(d->geom, d->geom + ng3 * 3 * d->n_elem);
  m->h_nbr.assign(d->neighbors, d->neighbors + 6 * (size_t)d->n_elem);
  m->h_ord.assign(d->orders, d->orders + 3 * (size_t)d->n_elem);
  dg_status st = build(m);
  if (st != DG_OK) {
    destroy_impl(m);
    return st;
  }
  *out = m;
  return DG_OK;
}

dg_status dg_mesh_destroy(dg_mesh* m) {
  if (!m) return DG_ERR_ARG;
  if (m->stream) cudaStreamSynchronize(m->stream);
  else cudaDeviceSynchronize();
  destroy_impl(m);
  return DG_OK;
}

dg_status dg_mesh_info(const dg_mesh* m, int64_t* n_nodes, int32_t* n_elem) {
  if (!m) return DG_ERR_ARG;
  if (n_nodes) *n_nodes = m->n_nodes;
  if (n_elem) *n_elem = m->n_elem;
  return DG_OK;
}

dg_status dg_mesh_layout(const dg_mesh* m, int64_t* n_nodes, const int64_t** elem_offset) {
  if (!m) return DG_ERR_ARG;
  if (n_nodes) *n_nodes = m->n_nodes;
  if (elem_offset) *elem_offset = m->d_off;
  return DG_OK;
}

dg_status dg_set_stream(dg_mesh* m, void* stream) {
  if (!m) return DG_ERR_ARG;
  m->stream = static_cast<cudaStream_t>(stream);
  for (auto* c : m->coarse) c->stream = m->stream;
  return DG_OK;
}

dg_status dg_node_coords(dg_mesh* m, double* xyz) {
  if (!m || !xyz) return DG_ERR_ARG;
  const int ng3 = (m->G + 1) * (m->G + 1) * (m->G + 1);
  std::vector<double> out(3 * (size_t)m->n_nodes);
#pragma omp parallel for schedule(dynamic, 64)
  for (int e = 0; e < m->n_elem; ++e) {
    std::vector<double> X, Ja, J;
    element_geometry(&m->h_geom[(size_t)e * ng3 * 3], m->G, &m->h_ord[3 * e], X, Ja, J);
    std::copy(X.begin(), X.end(), out.begin() + 3 * m->h_off[e]);
  }
  DG_CUDA(cudaMemcpy(xyz, out.data(), sizeof(double) * out.size(), cudaMemcpyHostToDevice));
  return DG_OK;
}

dg_status dg_residual(dg_mesh* m, const double* q, double* r, uint32_t flags) {
  if (!m || !q || !r || q == r || (flags & ~DG_ISOLATED)) return DG_ERR_ARG;
  return residual_impl(m, q, r, flags & DG_ISOLATED);
}

dg_status dg_max_dt(dg_mesh* m, const double* q, double cfl, double* dt_dev) {
  if (!m || !q || !dt_dev || !(cfl > 0.0)) return DG_ERR_ARG;
  return from_cuda(dgk::max_dt(m, q, cfl, dt_dev));
}

dg_status dg_rk_step(dg_mesh* m, double* q, double* g, const double* dt_dev) {
  if (!m || !q || !g || !dt_dev || q == g) return DG_ERR_ARG;
  if (m->faces_unsupported) return DG_ERR_UNSUPPORTED;
  return rk_step_impl(m, q, g, dt_dev, false);   // the caller may have changed q since the last step
}

dg_status dg_tau_estimate(dg_mesh* m, const double* q, const double* r_p, const int32_t* sweep, int32_t n_sweep,
                          uint32_t flags, void* map_new, void* map_trad) {
  if (!m || !q || !sweep || n_sweep <= 0 || (!map_new && !map_trad)) return DG_ERR_ARG;
  if (flags & ~(DG_TAU_ISOLATED | DG_TAU_FP32 | DG_TAU_ACCUM_MAX)) return DG_ERR_ARG;
  for (int s = 0; s < 3 * n_sweep; ++s)
    if (sweep[s] < 1 || sweep[s] > DG_MAX_ORDER) return DG_ERR_ARG;
  const bool fp32 = flags & DG_TAU_FP32, acc = flags & DG_TAU_ACCUM_MAX;
  if (flags & DG_TAU_ISOLATED) {
    int limit = 0;
    DG_CUDA(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
    if (dgk::tau_smem_bytes(m, fp32, limit) > (size_t)limit) return DG_ERR_UNSUPPORTED;
    dg_status st = build_tau_bank(m);
    if (st != DG_OK) return st;
    if (!r_p && fp32 && !m->d_rp32) DG_CUDA(cudaMalloc(&m->d_rp32, sizeof(float) * 5 * m->n_nodes));
    if (!r_p && !fp32 && !m->d_rp) DG_CUDA(cudaMalloc(&m->d_rp, sizeof(double) * 5 * m->n_nodes));
    std::vector<int32_t> hs(sweep, sweep + 3 * n_sweep);
    if (hs != m->h_sweep) {
      if (m->d_sweep) cudaFree(m->d_sweep);
      m->d_sweep = nullptr;
      DG_CUDA(upload(&m->d_sweep, hs.data(), hs.size()));
      m->h_sweep = hs;
      dg_status st2 = build_tau_units(m);
      if (st2 != DG_OK) return st2;
    }
    return from_cuda(dgk::tau_isolated(m, q, r_p, m->d_sweep, n_sweep, fp32, acc, map_new, map_trad));
  }
  // non-isolated: full residual of coarse discretisations with orders min(N, P_e)
  if (m->faces_unsupported) return DG_ERR_UNSUPPORTED;
  const double* rp = r_p;
  if (!rp) {
    if (!m->d_rp) DG_CUDA(cudaMalloc(&m->d_rp, sizeof(double) * 5 * m->n_nodes));
    dg_status st = residual_impl(m, q, m->d_rp, false);
    if (st != DG_OK) return st;
    rp = m->d_rp;
  }
  for (int s = 0; s < n_sweep; ++s) {
    const int32_t* N = sweep + 3 * s;
    dg_mesh_impl* c = nullptr;
    for (size_t i = 0; i < m->coarse.size(); ++i)
      if (m->coarse_key[3 * i] == N[0] && m->coarse_key[3 * i + 1] == N[1] && m->coarse_key[3 * i + 2] == N[2])
        c = m->coarse[i];
    if (!c) {
      std::vector<int32_t> co(m->h_ord.size());
      for (int e = 0; e < m->n_elem; ++e)
        for (int d = 0; d < 3; ++d) co[3 * e + d] = std::min(N[d], m->h_ord[3 * e + d]);
      dg_status st;
      c = make_child(m, co, &st);
      if (!c) return st;
      DG_CUDA(cudaMalloc(&c->d_qc, sizeof(double) * 5 * c->n_nodes));
      DG_CUDA(cudaMalloc(&c->d_rc, sizeof(double) * 5 * c->n_nodes));
      m->coarse.push_back(c);
      m->coarse_key.insert(m->coarse_key.end(), N, N + 3);
    }
    c->stream = m->stream;
    cudaError_t e;
    if ((e = dgk::project_orders(m, c->d_ord, c->d_off, q, c->d_qc, 1))) return from_cuda(e);
    dg_status st = residual_impl(c, c->d_qc, c->d_rc, false);
    if (st != DG_OK) return st;
    if ((e = dgk::tau_combine(m, c, rp, c->d_rc, s, n_sweep, sweep, fp32, acc, map_new, map_trad)))
      return from_cuda(e);
  }
  return DG_OK;
}

dg_status dg_set_orders(dg_mesh* m, const int32_t* new_orders, const double* q_old, double* q_new) {
  if (!m || !new_orders || !q_old || !q_new || q_old == q_new) return DG_ERR_ARG;
  int64_t nn = 0;
  if (dg_count_nodes(m->n_elem, new_orders, &nn) != DG_OK) return DG_ERR_ARG;
  std::vector<int32_t> no(new_orders, new_orders + 3 * (size_t)m->n_elem);
  dg_status st;
  // the new mesh's offsets, metrics, buckets and face lists are built on the
  // device (rebuild.cu); the host tiles them into work items and batches
  dg_mesh_impl* c = make_child(m, no, &st, true);
  if (!c) return st;
  cudaError_t e = dgk::project_orders(m, c->d_ord, c->d_off, q_old, q_new, 0);
  if (e == cudaSuccess) e = m->stream ? cudaStreamSynchronize(m->stream) : cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    destroy_impl(c);
    return from_cuda(e);
  }
  // swap the rebuilt structures into m; the old ones leave with c
  cudaStream_t s = m->stream;
  std::swap(*static_cast<dg_mesh_impl*>(m), *c);
  m->stream = s;
  std::swap(m->d_err, c->d_err);   // keep the sticky error word of the mesh
  m->tau_unit_mode = c->tau_unit_mode;
  destroy_impl(c);
  return DG_OK;
}

dg_status dg_step_host(dg_mesh* m, const double* q_in, double* q_out, double t0, double t_end, double cfl,
                       int64_t max_steps, const int32_t* sweep, int32_t n_sweep, uint32_t tau_flags, void* map_new,
                       void* map_trad, double* t_out) {
  if (!m || !q_in || !q_out || !sweep || n_sweep <= 0 || (!map_new && !map_trad)) return DG_ERR_ARG;
  int dev = -1;
  DG_CUDA(cudaGetDevice(&dev));
  if (dev != m->device) return DG_ERR_ARG;   // the device buffers are allocated on the current device
  const size_t nq = 5 * (size_t)m->n_nodes;
  const size_t mb = (size_t)m->n_elem * n_sweep * ((tau_flags & DG_TAU_FP32) ? sizeof(float) : sizeof(double));
  cudaStream_t s = m->stream;
  if (!m->d_hq) {
    DG_CUDA(cudaMalloc(&m->d_hq, sizeof(double) * nq));
    DG_CUDA(cudaMalloc(&m->d_hg, sizeof(double) * nq));
    DG_CUDA(cudaMalloc(&m->d_ht, sizeof(double)));
  }
  if (m->hmap_bytes != mb) {   // a new sweep size or precision: new maps, accumulation from 0
    if (m->d_hmap_new) cudaFree(m->d_hmap_new);
    if (m->d_hmap_trad) cudaFree(m->d_hmap_trad);
    m->d_hmap_new = m->d_hmap_trad = nullptr;
    m->hmap_bytes = 0;
    DG_CUDA(cudaMalloc(&m->d_hmap_new, mb));
    DG_CUDA(cudaMalloc(&m->d_hmap_trad, mb));
    DG_CUDA(cudaMemsetAsync(m->d_hmap_new, 0, mb, s));
    DG_CUDA(cudaMemsetAsync(m->d_hmap_trad, 0, mb, s));
    m->hmap_bytes = mb;
  }
  DG_CUDA(cudaMemcpyAsync(m->d_hq, q_in, sizeof(double) * nq, cudaMemcpyHostToDevice, s));
  DG_CUDA(cudaMemsetAsync(m->d_hg, 0, sizeof(double) * nq, s));
  DG_CUDA(cudaMemcpyAsync(m->d_ht, &t0, sizeof(double), cudaMemcpyHostToDevice, s));
  DG_CUDA(cudaStreamSynchronize(s));   // t0 lives on this call's stack
  dg_status st = dg_advance(m, m->d_hq, m->d_hg, m->d_ht, t_end, cfl, max_steps, 0, nullptr);
  if (st != DG_OK) return st;
  st = dg_tau_estimate(m, m->d_hq, nullptr, sweep, n_sweep, tau_flags, map_new ? m->d_hmap_new : nullptr,
                       map_trad ? m->d_hmap_trad : nullptr);
  if (st != DG_OK) return st;
  DG_CUDA(cudaMemcpyAsync(q_out, m->d_hq, sizeof(double) * nq, cudaMemcpyDeviceToHost, s));
  if (map_new) DG_CUDA(cudaMemcpyAsync(map_new, m->d_hmap_new, mb, cudaMemcpyDeviceToHost, s));
  if (map_trad) DG_CUDA(cudaMemcpyAsync(map_trad, m->d_hmap_trad, mb, cudaMemcpyDeviceToHost, s));
  double t = 0.0;
  if (t_out) DG_CUDA(cudaMemcpyAsync(&t, m->d_ht, sizeof(double), cudaMemcpyDeviceToHost, s));
  DG_CUDA(cudaStreamSynchronize(s));
  if (t_out) *t_out = t;
  return DG_OK;
}

dg_status dg_set_tau_units(dg_mesh* m, int32_t mode) {
  if (!m || mode < DG_TAU_UNITS_AUTO || mode > DG_TAU_UNITS_SPLIT) return DG_ERR_ARG;
  m->tau_unit_mode = mode;
  if (m->h_sweep.empty()) return DG_OK;
  // the next isolated sweep rebuilds the units for its list
  m->h_sweep.clear();
  return DG_OK;
}

dg_status dg_tau_units_info(const dg_mesh* m, int32_t max_classes, int32_t* n_classes, int32_t* n_units,
                            int32_t* n_shared) {
  if (!m || max_classes < 0 || !n_classes || (max_classes > 0 && (!n_units || !n_shared))) return DG_ERR_ARG;
  const int nc = m->h_sweep.empty() ? 0 : (int)m->tau_last_units.size();
  *n_classes = nc;
  for (int k = 0; k < nc && k < max_classes; ++k) {
    n_units[k] = m->tau_last_units[k];
    n_shared[k] = m->tau_last_shared[k];
  }
  return DG_OK;
}

static dg_status adjoint_ready(dg_mesh* m) {
  if (m->faces_unsupported) return DG_ERR_UNSUPPORTED;
  int limit = 0;
  DG_CUDA(cudaDeviceGetAttribute(&limit, cudaDevAttrMaxSharedMemoryPerBlockOptin, m->device));
  if (sizeof(double) * dgk::mortar_adj_smem_max(m) + 1024 > (size_t)limit) return DG_ERR_UNSUPPORTED;
  const size_t sf = (size_t)m->h_soff[m->n_elem];
  if (!m->d_sadj) DG_CUDA(cudaMalloc(&m->d_sadj, sizeof(double) * 5 * sf));
  if (!m->d_adjt) DG_CUDA(cudaMalloc(&m->d_adjt, sizeof(double) * 5 * (size_t)m->n_nodes));
  if (!m->d_force) DG_CUDA(cudaMalloc(&m->d_force, sizeof(double) * 3 * (size_t)std::max(m->n_faces, 1)));
  if (m->phys.eqs == DG_NAVIER_STOKES) {
    if (!m->d_gadj) DG_CUDA(cudaMalloc(&m->d_gadj, sizeof(double) * 15 * sf));
    if (!m->d_lS) DG_CUDA(cudaMalloc(&m->d_lS, sizeof(double) * 15 * sf));
    if (!m->d_lG) DG_CUDA(cudaMalloc(&m->d_lG, sizeof(double) * 15 * (size_t)m->n_nodes));
  }
  return DG_OK;
}

dg_status dg_residual_vjp(dg_mesh* m, const double* q, const double* v, double* out, double* qinf_adj) {
  if (!m || !q || !v || !out || out == q || out == v) return DG_ERR_ARG;
  dg_status st = adjoint_ready(m);
  if (st != DG_OK) return st;
  return from_cuda(dgk::residual_vjp(m, q, v, out, nullptr, false, qinf_adj));
}

dg_status dg_wall_force(dg_mesh* m, const double* q, int32_t tag, double* force_dev) {
  if (!m || !q || !force_dev || tag >= 0) return DG_ERR_ARG;
  // a forward quantity: the boundary faces and, for Navier-Stokes, the BR1
  // gradient (its mortars included); only the per-face partial sums are needed
  if (m->faces_unsupported) return DG_ERR_UNSUPPORTED;
  if (!m->d_force) DG_CUDA(cudaMalloc(&m->d_force, sizeof(double) * 3 * (size_t)std::max(m->n_faces, 1)));
  return from_cuda(dgk::wall_force(m, q, tag, force_dev));
}

dg_status dg_wall_force_vjp(dg_mesh* m, const double* q, int32_t tag, const double* lam_dev, double* out,
                            const double* scale_dev) {
  if (!m || !q || !lam_dev || !out || out == q || tag >= 0) return DG_ERR_ARG;
  dg_status st = adjoint_ready(m);
  if (st != DG_OK) return st;
  return from_cuda(dgk::wall_force_vjp(m, q, tag, lam_dev, out, scale_dev));
}

dg_status dg_rk_step_vjp(dg_mesh* m, const double* q0, const double* dt_dev, double* lam, double* qinf_adj) {
  if (!m || !q0 || !dt_dev || !lam || lam == q0) return DG_ERR_ARG;
  dg_status st = adjoint_ready(m);
  if (st != DG_OK) return st;
  const size_t ns = 5 * (size_t)m->n_nodes;
  if (!m->d_adjw) DG_CUDA(cudaMalloc(&m->d_adjw, sizeof(double) * 4 * ns));
  double* Q1 = m->d_adjw;
  double* Q2 = Q1 + ns;
  double* G = Q2 + ns;
  double* LG = G + ns;
  static const double A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
  static const double B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};
  cudaError_t e;
  // the stage states Q1, Q2 again, from q0 (the register starts at zero; the
  // first stage does not read it)
  if ((e = cudaMemcpyAsync(Q1, q0, sizeof(double) * ns, cudaMemcpyDeviceToDevice, m->stream))) return from_cuda(e);
  for (int k = 0; k < 2; ++k) {
    double* Qk = k ? Q2 : Q1;
    if (k && (e = cudaMemcpyAsync(Q2, Q1, sizeof(double) * ns, cudaMemcpyDeviceToDevice, m->stream)))
      return from_cuda(e);
    if (m->phys.eqs == DG_NAVIER_STOKES) {   // BR1 gradient of the stage state, as in dg_rk_step
      if ((e = dgk::face_qhat(m, Qk))) return from_cuda(e);
      if ((e = dgk::gradient(m, Qk, m->d_grad, false))) return from_cuda(e);
    }
    if ((e = dgk::face_flux(m, Qk, m->d_grad, false))) return from_cuda(e);
    if ((e = dgk::volume(m, Qk, m->d_grad, nullptr, false, k, Qk, G, dt_dev))) return from_cuda(e);
  }
  // reversed: with G_k = A_k G_{k-1} + dt R(Q_{k-1}) and Q_k = Q_{k-1} + B_k G_k,
  //   LG = B3 lam;            lam += dt J(Q2)^T LG
  //   LG = A3 LG + B2 lam;    lam += dt J(Q1)^T LG
  //   LG = A2 LG + B1 lam;    lam += dt J(q0)^T LG
  const double* Qs[3] = {q0, Q1, Q2};
  for (int k = 2; k >= 0; --k) {
    const double a = k == 2 ? 0.0 : A[k + 1], b = B[k];
    if ((e = dgk::axpby(m, LG, lam, a, b, (int64_t)ns))) return from_cuda(e);
    if ((e = dgk::residual_vjp(m, Qs[k], LG, lam, dt_dev, true, qinf_adj))) return from_cuda(e);
  }
  return DG_OK;
}

dg_status dg_get_error(dg_mesh* m) {
  if (!m) return DG_ERR_ARG;
  cudaError_t e = m->stream ? cudaStreamSynchronize(m->stream) : cudaDeviceSynchronize();
  if (e) return from_cuda(e);
  unsigned w = 0;
  DG_CUDA(cudaMemcpy(&w, m->d_err, sizeof(w), cudaMemcpyDeviceToHost));
  DG_CUDA(cudaMemset(m->d_err, 0, sizeof(unsigned)));
  if (w & 2u) return DG_ERR_INDEX;
  return w ? DG_ERR_NONPHYSICAL : DG_OK;
}

dg_status dg_debug_set_index(dg_mesh* m, int32_t list, int64_t i, int32_t value, int32_t* old_value) {
#ifdef DG_BOUNDS_CHECK
  if (!m || i < 0) return DG_ERR_ARG;
  int32_t* base = nullptr;
  int64_t len = 0;
  switch (list) {
    case DG_LIST_VOLUME_ELEMENTS: base = m->d_velist; len = m->n_elem; break;
    case DG_LIST_TAU_ELEMENTS: base = m->d_elist; len = m->n_elem; break;
    case DG_LIST_FACE_LEFT: {   // the L field (the first) of face record i
      constexpr int64_t words = sizeof(FaceRec) / sizeof(int32_t);
      if (i >= m->n_faces) return DG_ERR_ARG;
      base = reinterpret_cast<int32_t*>(m->d_faces);
      len = (int64_t)m->n_faces * words;
      i *= words;
      break;
    }
    case DG_LIST_MORTAR_FACES: base = m->d_mfaces; len = 3 * (int64_t)m->n_mfaces; break;
    default: return DG_ERR_ARG;
  }
  if (!base || i >= len) return DG_ERR_ARG;
  DG_CUDA(m->stream ? cudaStreamSynchronize(m->stream) : cudaDeviceSynchronize());
  if (old_value) DG_CUDA(cudaMemcpy(old_value, base + i, sizeof(int32_t), cudaMemcpyDeviceToHost));
  DG_CUDA(cudaMemcpy(base + i, &value, sizeof(int32_t), cudaMemcpyHostToDevice));
  return DG_OK;
#else
  (void)list;
  (void)i;
  (void)value;
  (void)old_value;
  return m ? DG_ERR_UNSUPPORTED : DG_ERR_ARG;
#endif
}

}  // extern "C"
