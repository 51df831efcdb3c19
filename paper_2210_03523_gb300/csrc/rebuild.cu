// rebuild.cu -- the order-dependent parts of a mesh built on the device: the
// node and face-node offsets, the curved elements' metrics at their orders
// (and at every coarse order of the isolated tau sweep), the elements
// bucketed by order triple, and the faces classified (conforming,
// p-nonconforming, boundary) and grouped by mortar shape.  dg_set_orders
// (Sec. 2.4: the mesh changes after every adaptation stage of the dynamic
// strategy, Fig. 1) rebuilds its mesh this way; the host then cuts the sorted
// buckets and shape groups into tiles and batches from copies of the sorted
// lists.
#include <cuda_runtime.h>

#include <algorithm>
#include <cub/device/device_radix_sort.cuh>
#include <cub/device/device_scan.cuh>
#include <vector>

#include "dg_internal.h"

namespace {

constexpr int kGeomThreads = 256;

// Per-order 1D tables of the metric construction (indexed by the order N,
// 1..DG_MAX_ORDER; a job's node count n = N + 1 reads entry n - 1): E[N] ((N+1) x (G+1))
// interpolates the equispaced geometry lattice of order G to the order-N GL
// nodes, D[N] ((N+1) x (N+1)) is the GL derivative matrix.
struct GeomTabOff {
  int E[DG_NP1];
  int D[DG_NP1];
};


// out[i + eo0 (j + eo1 k)] = sum_mm A[r nf + mm] in[... + mm stride]: the
// host's tensor_apply with the same summation order and roundings (no
// contraction), so that both builds give the same bits.
__device__ __forceinline__ double apply_at(const double* __restrict__ A, int nf, int dir, const int ext[3],
                                           const double* in, int i, int j, int k) {
  const int stride = dir == 0 ? 1 : (dir == 1 ? ext[0] : ext[0] * ext[1]);
  const int r = dir == 0 ? i : (dir == 1 ? j : k);
  const int ii = dir == 0 ? 0 : i, jj = dir == 1 ? 0 : j, kk = dir == 2 ? 0 : k;
  const double* src = in + ii + ext[0] * (jj + ext[1] * kk);
  const double* a = A + r * nf;
  double s = 0.0;
  for (int mm = 0; mm < nf; ++mm) s = __dadd_rn(s, __dmul_rn(a[mm], src[mm * stride]));
  return s;
}

// the whole array: out has ext with ext[dir] replaced by nt
__device__ void apply_dir(const double* A, int nt, int nf, int dir, const int ext[3], const double* in, double* out) {
  int eo[3] = {ext[0], ext[1], ext[2]};
  eo[dir] = nt;
  const int tot = eo[0] * eo[1] * eo[2];
  for (int t = threadIdx.x; t < tot; t += blockDim.x) {
    const int i = t % eo[0], jk = t / eo[0], j = jk % eo[1], k = jk / eo[1];
    out[t] = apply_at(A, nf, dir, ext, in, i, j, k);
  }
}

// Metrics of a curved element at orders N, Kopriva's conservative curl form
// (J a^i_n = -e_i . curl_xi(I^N(X_l grad_xi X_m)), (n, m, l) cyclic), as the
// host construction computes them: the element map through the geometry
// lattice interpolated to the GL nodes, its GL derivatives, J the triple
// product, then the curl of X_l grad X_m.  One CTA a job; bad |= 1 where a
// Jacobian is not positive.
__global__ void __launch_bounds__(kGeomThreads) geom_kernel(const double* __restrict__ geom, int G,
                                                            const double* __restrict__ tab, GeomTabOff toff,
                                                            const DgGeomJob* __restrict__ jobs, int n_jobs,
                                                            int fields, double* out, float* out32, unsigned* bad) {
  extern __shared__ double gsm[];
  const int ng = G + 1, ng3 = ng * ng * ng;
  for (int jb = blockIdx.x; jb < n_jobs; jb += gridDim.x) {
    const DgGeomJob J = jobs[jb];
    const int n1 = J.n1, n2 = J.n2, n3 = J.n3, n = n1 * n2 * n3;
    const int nn3[3] = {n1, n2, n3};
    double* Xg = gsm;                    // [3][ng^3] the lattice
    double* t1 = Xg + 3 * ng3;           // [n1 ng ng]
    double* t2 = t1 + DG_NP1 * ng * ng;  // [n1 n2 ng]
    double* X = t2 + DG_NP1 * DG_NP1 * ng;   // [3][n]
    double* dX = X + 3 * n;              // [(c 3 + i)][n] = dX_c / dxi_i
    double* W = dX + 9 * n;              // [3][n]
    const double* gn = geom + (size_t)J.e * ng3 * 3;
    for (int t = threadIdx.x; t < 3 * ng3; t += blockDim.x) {
      const int c = t / ng3, p = t - c * ng3;
      Xg[t] = gn[3 * p + c];
    }
    __syncthreads();
    for (int c = 0; c < 3; ++c) {
      int ext[3] = {ng, ng, ng};
      apply_dir(tab + toff.E[n1 - 1], n1, ng, 0, ext, Xg + c * ng3, t1);
      __syncthreads();
      ext[0] = n1;
      apply_dir(tab + toff.E[n2 - 1], n2, ng, 1, ext, t1, t2);
      __syncthreads();
      ext[1] = n2;
      apply_dir(tab + toff.E[n3 - 1], n3, ng, 2, ext, t2, X + c * n);
      __syncthreads();
    }
    const int ext[3] = {n1, n2, n3};
    for (int t = threadIdx.x; t < 9 * n; t += blockDim.x) {
      const int ci = t / n, p = t - ci * n, c = ci / 3, i = ci - 3 * c;
      const int x = p % n1, yz = p / n1, y = yz % n2, z = yz / n2;
      dX[t] = apply_at(tab + toff.D[nn3[i] - 1], nn3[i], i, ext, X + c * n, x, y, z);
    }
    __syncthreads();
    double* o = out + J.out;
    float* o32 = out32 ? out32 + J.out : nullptr;
    for (int p = threadIdx.x; p < n; p += blockDim.x) {
      auto g = [&](int c, int i) { return dX[(c * 3 + i) * n + p]; };
      const double a = __dmul_rn(g(0, 0), __dsub_rn(__dmul_rn(g(1, 1), g(2, 2)), __dmul_rn(g(1, 2), g(2, 1))));
      const double b = __dmul_rn(g(0, 1), __dsub_rn(__dmul_rn(g(1, 0), g(2, 2)), __dmul_rn(g(1, 2), g(2, 0))));
      const double c = __dmul_rn(g(0, 2), __dsub_rn(__dmul_rn(g(1, 0), g(2, 1)), __dmul_rn(g(1, 1), g(2, 0))));
      const double Jp = __dadd_rn(__dsub_rn(a, b), c);
      if (!(Jp > 0.0)) atomicOr(bad, 1u);
      o[9 * n + p] = Jp;
      if (fields == 11) o[10 * n + p] = 1.0 / Jp;
      if (o32) o32[9 * n + p] = (float)Jp;
    }
    for (int nn = 0; nn < 3; ++nn) {
      const int mm = (nn + 1) % 3, ll = (nn + 2) % 3;
      for (int t = threadIdx.x; t < 3 * n; t += blockDim.x) {
        const int jd = t / n, p = t - jd * n;
        W[t] = __dmul_rn(X[ll * n + p], dX[(mm * 3 + jd) * n + p]);
      }
      __syncthreads();
      for (int t = threadIdx.x; t < 3 * n; t += blockDim.x) {
        const int i = t / n, p = t - i * n, i1 = (i + 1) % 3, i2 = (i + 2) % 3;
        const int x = p % n1, yz = p / n1, y = yz % n2, z = yz / n2;
        // (curl W)_i = d_i1 W_i2 - d_i2 W_i1;  J a^i_nn = -(curl W)_i
        const double s1 = apply_at(tab + toff.D[nn3[i1] - 1], nn3[i1], i1, ext, W + i2 * n, x, y, z);
        const double s2 = apply_at(tab + toff.D[nn3[i2] - 1], nn3[i2], i2, ext, W + i1 * n, x, y, z);
        const double v = __dadd_rn(__dsub_rn(0.0, s1), s2);
        o[(i * 3 + nn) * n + p] = v;
        if (o32) o32[(i * 3 + nn) * n + p] = (float)v;
      }
      __syncthreads();
    }
  }
}

size_t geom_smem_bytes(int G, int n_max) {
  const int ng = G + 1;
  return sizeof(double) * ((size_t)3 * ng * ng * ng + (size_t)DG_NP1 * ng * ng + (size_t)DG_NP1 * DG_NP1 * ng +
                           15 * (size_t)n_max);
}

// The tables for geometry order G, from the same host routines the host
// construction uses.
void geom_tables(int G, GeomTabOff* off, std::vector<double>* tab) {
  const int ng = G + 1;
  double xs[DG_NP1 + 8];
  for (int a = 0; a <= G; ++a) xs[a] = -1.0 + 2.0 * a / G;
  tab->clear();
  for (int N = 1; N <= DG_MAX_ORDER; ++N) {
    double x[DG_NP1], w[DG_NP1], E[DG_NP1 * 16], D[DG_NP1 * DG_NP1];
    dgb::gl_nodes_weights(N, x, w);
    dgb::interp_matrix(xs, ng, x, N + 1, E);
    dgb::deriv_matrix(N, D);
    off->E[N] = (int)tab->size();
    tab->insert(tab->end(), E, E + (N + 1) * ng);
    off->D[N] = (int)tab->size();
    tab->insert(tab->end(), D, D + (N + 1) * (N + 1));
  }
}

}  // namespace

// Metrics of every job into out (and out32), on the mesh's stream; the
// lattice of every element at d_geom.  Returns DG_ERR_ARG for a Jacobian that
// is not positive.
dg_status dg_device_metrics(dg_mesh_impl* m, const std::vector<DgGeomJob>& jobs, int fields, double* out,
                            float* out32) {
  const int n_jobs = (int)jobs.size();
  if (n_jobs == 0) return DG_OK;
  if (m->G + 1 > 16 || !m->d_geom) return DG_ERR_UNSUPPORTED;
  GeomTabOff toff;
  std::vector<double> tab;
  geom_tables(m->G, &toff, &tab);
  int n_max = 1;
  for (const auto& j : jobs) n_max = std::max(n_max, j.n1 * j.n2 * j.n3);
  double* d_tab = nullptr;
  DgGeomJob* d_jobs = nullptr;
  unsigned* d_bad = nullptr;
  cudaError_t e = cudaMalloc(&d_tab, sizeof(double) * tab.size());
  if (!e) e = cudaMalloc(&d_jobs, sizeof(DgGeomJob) * jobs.size());
  if (!e) e = cudaMalloc(&d_bad, sizeof(unsigned));
  if (!e) e = cudaMemcpyAsync(d_tab, tab.data(), sizeof(double) * tab.size(), cudaMemcpyHostToDevice, m->stream);
  if (!e) e = cudaMemcpyAsync(d_jobs, jobs.data(), sizeof(DgGeomJob) * jobs.size(), cudaMemcpyHostToDevice, m->stream);
  if (!e) e = cudaMemsetAsync(d_bad, 0, sizeof(unsigned), m->stream);
  const size_t smem = geom_smem_bytes(m->G, n_max);
  if (!e) e = cudaFuncSetAttribute(geom_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  unsigned bad = 0;
  if (!e) {
    const int grid = std::min(n_jobs, 152 * 8);
    geom_kernel<<<grid, kGeomThreads, smem, m->stream>>>(m->d_geom, m->G, d_tab, toff, d_jobs, n_jobs, fields, out,
                                                         out32, d_bad);
    e = cudaGetLastError();
  }
  if (!e) e = cudaMemcpyAsync(&bad, d_bad, sizeof(unsigned), cudaMemcpyDeviceToHost, m->stream);
  if (!e) e = cudaStreamSynchronize(m->stream);
  cudaFree(d_tab);
  cudaFree(d_jobs);
  cudaFree(d_bad);
  if (e) return e == cudaErrorMemoryAllocation ? DG_ERR_NOMEM : DG_ERR_CUDA;
  return bad ? DG_ERR_ARG : DG_OK;
}

// ---------------------------------------------------------------------------
// Offsets, buckets and faces
// ---------------------------------------------------------------------------
namespace {

constexpr int kListThreads = 256;
constexpr uint32_t kFaceNone = (1u << 18) - 1;   // a candidate slot that holds no face (sorts last)
constexpr int kFaceKeyBits = 18;

// Per element: its bucket key (the order triple, N1 slowest, as the host's
// ordered map of triples), node and face-node counts; thread ne writes the
// zero after the last element, so that an exclusive scan gives the offsets.
__global__ void elem_lists_kernel(const int32_t* __restrict__ ord, int ne, uint32_t* key, int32_t* idx, int64_t* cn,
                                  int64_t* cs) {
  const int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e > ne) return;
  if (e == ne) {
    cn[ne] = 0;
    cs[ne] = 0;
    return;
  }
  const int N1 = ord[3 * e], N2 = ord[3 * e + 1], N3 = ord[3 * e + 2];
  const int64_t a = N1 + 1, b = N2 + 1, c = N3 + 1;
  key[e] = (uint32_t)(((N1 - 1) * 8 + (N2 - 1)) * 8 + (N3 - 1));
  idx[e] = e;
  cn[e] = a * b * c;
  cs[e] = 2 * (b * c + a * c + a * b);
}

// Candidate face slot s = 6 e + f of element e: an interior face is listed by
// its -xi side (f odd, the neighbour across face f holds face f - 1), a
// boundary face by its element.  Keys: 0 a conforming face of the warp list,
// 2 a boundary face, 4 + 4 sig + dir a face of the shape batches (the
// p-nonconforming ones, and on affine Euler meshes the conforming ones too),
// sig = ((la 16 + lb) 16 + ra) 16 + rb the tangential node counts of both
// sides.  counts[kind] += 1 for kinds 0 (conforming), 1 (p-nonconforming), 2.
__global__ void face_keys_kernel(const int32_t* __restrict__ ord, const int32_t* __restrict__ nbr, int ne,
                                 int batch_conf, uint32_t* key, int32_t* idx, int* counts) {
  const int s = blockIdx.x * blockDim.x + threadIdx.x;
  if (s >= 6 * ne) return;
  const int e = s / 6, f = s - 6 * e, d = f >> 1, side = f & 1, nb = nbr[s];
  const int t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
  uint32_t k = kFaceNone;
  if (nb >= 0) {
    if (side) {
      const int la = ord[3 * e + t0] + 1, lb = ord[3 * e + t1] + 1, ra = ord[3 * nb + t0] + 1,
                rb = ord[3 * nb + t1] + 1;
      const int kind = (la == ra && lb == rb) ? 0 : 1;
      atomicAdd(counts + kind, 1);
      if (kind == 1 || batch_conf) k = 4u + 4u * (uint32_t)(((la * 16 + lb) * 16 + ra) * 16 + rb) + (uint32_t)d;
      else k = 0;
    }
  } else {
    k = 2;
    atomicAdd(counts + 2, 1);
  }
  key[s] = k;
  idx[s] = s;
}

// The warp-list faces (sorted positions [0, n)) as face records, and the face
// node count of each (count[n] = 0 for the scan).
__global__ void warp_faces_kernel(const uint32_t* __restrict__ ks, const int32_t* __restrict__ ss, int n,
                                  const int32_t* __restrict__ ord, const int32_t* __restrict__ nbr, FaceRec* faces,
                                  int64_t* count) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i > n) return;
  if (i == n) {
    count[n] = 0;
    return;
  }
  const int s = ss[i], e = s / 6, f = s - 6 * e, d = f >> 1;
  const int t0 = d == 0 ? 1 : 0, t1 = d == 2 ? 1 : 2;
  faces[i] = ks[i] == 0 ? FaceRec{e, nbr[s], d, 0} : FaceRec{e, nbr[s], f, 2};
  count[i] = (int64_t)(ord[3 * e + t0] + 1) * (ord[3 * e + t1] + 1);
}

// (face, node) of every node of the warp-list faces
__global__ void face_nodes_kernel(const int64_t* __restrict__ start, int n, int32_t* fnodes) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int64_t a = start[i], b = start[i + 1];
  for (int64_t p = a; p < b; ++p) {
    fnodes[2 * p] = i;
    fnodes[2 * p + 1] = (int32_t)(p - a);
  }
}

// The batched faces (sorted positions [first, first + n)) as [L, R, dir] and
// their shape signatures.
__global__ void batched_faces_kernel(const uint32_t* __restrict__ ks, const int32_t* __restrict__ ss, int first,
                                     int n, const int32_t* __restrict__ nbr, int32_t* mf, int32_t* sig) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int s = ss[first + i], e = s / 6, f = s - 6 * e;
  mf[3 * i] = e;
  mf[3 * i + 1] = nbr[s];
  mf[3 * i + 2] = f >> 1;
  sig[i] = (int32_t)((ks[first + i] - 4u) >> 2);
}

int blocks_for(int64_t n) { return (int)((n + kListThreads - 1) / kListThreads); }

// device scratch freed on every return path
struct Scratch {
  std::vector<void*> p;
  template <typename T>
  cudaError_t get(T** out, size_t n) {
    void* v = nullptr;
    cudaError_t e = cudaMalloc(&v, (n ? n : 1) * sizeof(T));
    if (!e) p.push_back(v);
    *out = static_cast<T*>(v);
    return e;
  }
  ~Scratch() {
    for (void* v : p) cudaFree(v);
  }
};

template <typename K, typename V>
cudaError_t sort_pairs(Scratch& sc, const K* kin, K* kout, const V* vin, V* vout, int n, int bits, cudaStream_t st) {
  size_t tb = 0;
  cudaError_t e = cub::DeviceRadixSort::SortPairs(nullptr, tb, kin, kout, vin, vout, n, 0, bits, st);
  void* tmp = nullptr;
  if (!e) e = sc.get(reinterpret_cast<char**>(&tmp), tb);
  if (!e) e = cub::DeviceRadixSort::SortPairs(tmp, tb, kin, kout, vin, vout, n, 0, bits, st);
  return e;
}

cudaError_t excl_sum(Scratch& sc, const int64_t* in, int64_t* out, int n, cudaStream_t st) {
  size_t tb = 0;
  cudaError_t e = cub::DeviceScan::ExclusiveSum(nullptr, tb, in, out, n, st);
  void* tmp = nullptr;
  if (!e) e = sc.get(reinterpret_cast<char**>(&tmp), tb);
  if (!e) e = cub::DeviceScan::ExclusiveSum(tmp, tb, in, out, n, st);
  return e;
}

}  // namespace

// The order-dependent lists of a mesh whose d_ord and d_nbr are on the
// device: d_off, d_soff (and their host copies), the warp-list faces d_faces
// with their nodes d_fnodes, and, copied to the host for the tiling, the
// elements sorted by order triple and the batched faces sorted by shape, then
// direction (element order kept within equal keys, as the host construction
// orders them).
dg_status dg_device_lists(dg_mesh_impl* m, bool batch_conforming, DgDeviceLists* out) {
  const int ne = m->n_elem;
  cudaStream_t st = m->stream;
  Scratch sc;
  uint32_t *ek = nullptr, *eks = nullptr, *fk = nullptr, *fks = nullptr;
  int32_t *ei = nullptr, *eis = nullptr, *fi = nullptr, *fis = nullptr, *cnt = nullptr;
  int64_t *cn = nullptr, *cs = nullptr;
  cudaError_t e = cudaSuccess;
  auto ok = [&](cudaError_t x) { if (!e) e = x; return !e; };
  ok(sc.get(&ek, ne)); ok(sc.get(&eks, ne)); ok(sc.get(&ei, ne)); ok(sc.get(&eis, ne));
  ok(sc.get(&cn, ne + 1)); ok(sc.get(&cs, ne + 1));
  ok(sc.get(&fk, 6 * (size_t)ne)); ok(sc.get(&fks, 6 * (size_t)ne)); ok(sc.get(&fi, 6 * (size_t)ne));
  ok(sc.get(&fis, 6 * (size_t)ne)); ok(sc.get(&cnt, 3));
  if (m->d_off) cudaFree(m->d_off);
  if (m->d_soff) cudaFree(m->d_soff);
  m->d_off = m->d_soff = nullptr;
  ok(cudaMalloc(&m->d_off, sizeof(int64_t) * (ne + 1)));
  ok(cudaMalloc(&m->d_soff, sizeof(int64_t) * (ne + 1)));
  if (e) return e == cudaErrorMemoryAllocation ? DG_ERR_NOMEM : DG_ERR_CUDA;
  // offsets and buckets
  elem_lists_kernel<<<blocks_for(ne + 1), kListThreads, 0, st>>>(m->d_ord, ne, ek, ei, cn, cs);
  ok(cudaGetLastError());
  ok(excl_sum(sc, cn, m->d_off, ne + 1, st));
  ok(excl_sum(sc, cs, m->d_soff, ne + 1, st));
  ok(sort_pairs(sc, ek, eks, ei, eis, ne, 9, st));
  // faces
  ok(cudaMemsetAsync(cnt, 0, 3 * sizeof(int), st));
  face_keys_kernel<<<blocks_for(6 * (int64_t)ne), kListThreads, 0, st>>>(m->d_ord, m->d_nbr, ne,
                                                                          batch_conforming ? 1 : 0, fk, fi, cnt);
  ok(cudaGetLastError());
  ok(sort_pairs(sc, fk, fks, fi, fis, 6 * ne, kFaceKeyBits, st));
  int kinds[3] = {0, 0, 0};
  out->off.resize(ne + 1);
  out->soff.resize(ne + 1);
  out->bucket_key.resize(ne);
  out->bucket_elems.resize(ne);
  ok(cudaMemcpyAsync(kinds, cnt, sizeof(kinds), cudaMemcpyDeviceToHost, st));
  ok(cudaMemcpyAsync(out->off.data(), m->d_off, sizeof(int64_t) * (ne + 1), cudaMemcpyDeviceToHost, st));
  ok(cudaMemcpyAsync(out->soff.data(), m->d_soff, sizeof(int64_t) * (ne + 1), cudaMemcpyDeviceToHost, st));
  ok(cudaMemcpyAsync(out->bucket_key.data(), eks, sizeof(int32_t) * ne, cudaMemcpyDeviceToHost, st));
  ok(cudaMemcpyAsync(out->bucket_elems.data(), eis, sizeof(int32_t) * ne, cudaMemcpyDeviceToHost, st));
  ok(cudaStreamSynchronize(st));
  if (e) return DG_ERR_CUDA;
  out->n_conf = kinds[0];
  out->n_mortar = kinds[1];
  out->n_bnd = kinds[2];
  const int n_warp = (batch_conforming ? 0 : kinds[0]) + kinds[2];
  const int n_batched = kinds[1] + (batch_conforming ? kinds[0] : 0);
  // the warp list and its face nodes
  int64_t* fcount = nullptr;
  int64_t* fstart = nullptr;
  ok(sc.get(&fcount, n_warp + 1));
  ok(sc.get(&fstart, n_warp + 1));
  if (m->d_faces) cudaFree(m->d_faces);
  if (m->d_fnodes) cudaFree(m->d_fnodes);
  m->d_faces = nullptr;
  m->d_fnodes = nullptr;
  ok(cudaMalloc(&m->d_faces, sizeof(FaceRec) * (n_warp ? n_warp : 1)));
  if (e) return DG_ERR_NOMEM;
  warp_faces_kernel<<<blocks_for(n_warp + 1), kListThreads, 0, st>>>(fks, fis, n_warp, m->d_ord, m->d_nbr,
                                                                      m->d_faces, fcount);
  ok(cudaGetLastError());
  ok(excl_sum(sc, fcount, fstart, n_warp + 1, st));
  int64_t n_fnodes = 0;
  ok(cudaMemcpyAsync(&n_fnodes, fstart + n_warp, sizeof(int64_t), cudaMemcpyDeviceToHost, st));
  ok(cudaStreamSynchronize(st));
  if (e) return DG_ERR_CUDA;
  ok(cudaMalloc(&m->d_fnodes, sizeof(int32_t) * 2 * (n_fnodes ? n_fnodes : 1)));
  if (e) return DG_ERR_NOMEM;
  if (n_warp) face_nodes_kernel<<<blocks_for(n_warp), kListThreads, 0, st>>>(fstart, n_warp, m->d_fnodes);
  ok(cudaGetLastError());
  m->n_faces = n_warp;
  m->n_fnodes = (int)n_fnodes;
  // the batched faces, to the host for the shape groups and their batches
  int32_t *mf = nullptr, *sg = nullptr;
  ok(sc.get(&mf, 3 * (size_t)n_batched));
  ok(sc.get(&sg, n_batched));
  if (n_batched)
    batched_faces_kernel<<<blocks_for(n_batched), kListThreads, 0, st>>>(fks, fis, n_warp, n_batched, m->d_nbr, mf,
                                                                          sg);
  ok(cudaGetLastError());
  out->mfaces.resize(3 * (size_t)n_batched);
  out->msig.resize(n_batched);
  ok(cudaMemcpyAsync(out->mfaces.data(), mf, sizeof(int32_t) * 3 * n_batched, cudaMemcpyDeviceToHost, st));
  ok(cudaMemcpyAsync(out->msig.data(), sg, sizeof(int32_t) * n_batched, cudaMemcpyDeviceToHost, st));
  ok(cudaStreamSynchronize(st));
  return e ? DG_ERR_CUDA : DG_OK;
}
