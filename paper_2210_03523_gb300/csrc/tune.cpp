// tune.cpp -- the tile-shape autotuner (dg_autotune) and the tile budgets
// (dg_get_tiles, dg_set_tiles).  Elements of mixed anisotropic orders run in
// one launch bucketed by (N1,N2,N3) (Sec. 2.4); this picks, per element-size
// and mortar-size class, the node budget of a CTA's tile by timing the
// kernels on the mesh itself.
#include <cuda_runtime.h>

#include <algorithm>
#include <vector>

#include "dg_internal.h"

namespace {

constexpr int kCandidates[] = {64, 128, 192, 256, 384, 512};   // nodes per tile / mortar nodes per batch
constexpr int kNumCand = sizeof(kCandidates) / sizeof(kCandidates[0]);

dg_status status_of(cudaError_t e) {
  return e == cudaSuccess ? DG_OK : e == cudaErrorMemoryAllocation ? DG_ERR_NOMEM : DG_ERR_CUDA;
}

// median time (ms) of reps launches of fn on the mesh stream, after one warm-up
template <typename F>
dg_status time_launch(dg_mesh_impl* m, int reps, F fn, double* ms) {
  cudaEvent_t a = nullptr, b = nullptr;
  cudaError_t e;
  if ((e = cudaEventCreate(&a)) || (e = cudaEventCreate(&b))) {
    if (a) cudaEventDestroy(a);
    return status_of(e);
  }
  std::vector<float> t;
  e = fn();
  for (int r = 0; e == cudaSuccess && r < reps; ++r) {
    float x = 0.f;
    if ((e = cudaEventRecord(a, m->stream)) || (e = fn()) || (e = cudaEventRecord(b, m->stream)) ||
        (e = cudaEventSynchronize(b)) || (e = cudaEventElapsedTime(&x, a, b)))
      break;
    t.push_back(x);
  }
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  if (e) return status_of(e);
  std::sort(t.begin(), t.end());
  *ms = t.empty() ? 0.0 : t[t.size() / 2];
  return DG_OK;
}

// time of the production launches on the current work lists: the volume
// residual (every tile class) and the face fluxes (mortar batches included)
dg_status time_volume(dg_mesh_impl* m, const double* q, double* r, int reps, double* ms) {
  return time_launch(m, reps, [&]() { return dgk::volume(m, q, m->d_grad, r, false, -1, nullptr, nullptr, nullptr); },
                     ms);
}
dg_status time_faces(dg_mesh_impl* m, const double* q, int reps, double* ms) {
  return time_launch(m, reps, [&]() { return dgk::face_flux(m, q, m->d_grad, false); }, ms);
}

dg_status rebuild(dg_mesh_impl* m) {
  dg_advance_release(m);   // the graphs hold the old work lists
  dg_status st = build_volume_items(m);
  if (st == DG_OK) st = build_mortar_batches(m);
  return st;
}

void fill_budgets(const dg_mesh_impl* m, dg_tiles* out) {
  for (int k = 0; k < kSizeClasses; ++k) {
    out->vol_budget[k] = m->vol_budget[k];
    out->mortar_budget[k] = m->mortar_budget[k];
    out->vol_ms[k] = out->vol_ms_default[k] = out->mortar_ms[k] = out->mortar_ms_default[k] = -1.0;
  }
}

}  // namespace

extern "C" dg_status dg_get_tiles(const dg_mesh* mesh, dg_tiles* out) {
  if (!mesh || !out) return DG_ERR_ARG;
  fill_budgets(mesh, out);
  return DG_OK;
}

extern "C" dg_status dg_set_tiles(dg_mesh* mesh, const dg_tiles* in) {
  dg_mesh_impl* m = mesh;
  if (!m || !in) return DG_ERR_ARG;
  for (int k = 0; k < kSizeClasses; ++k)
    if (in->vol_budget[k] < 1 || in->vol_budget[k] > DG_MAX_VOL_BUDGET || in->mortar_budget[k] < 1 ||
        in->mortar_budget[k] > DG_MAX_MORTAR_BUDGET)
      return DG_ERR_ARG;
  dg_status st = status_of(m->stream ? cudaStreamSynchronize(m->stream) : cudaDeviceSynchronize());
  if (st != DG_OK) return st;
  std::copy(in->vol_budget, in->vol_budget + kSizeClasses, m->vol_budget);
  std::copy(in->mortar_budget, in->mortar_budget + kSizeClasses, m->mortar_budget);
  return rebuild(m);
}

extern "C" dg_status dg_autotune(dg_mesh* mesh, const double* q, int32_t reps, dg_tiles* out) {
  dg_mesh_impl* m = mesh;
  if (!m || !q || reps < 1 || reps > 1000) return DG_ERR_ARG;
  if (m->faces_unsupported) return DG_ERR_UNSUPPORTED;
  cudaError_t e = m->stream ? cudaStreamSynchronize(m->stream) : cudaDeviceSynchronize();
  if (e) return status_of(e);
  // which classes have elements / mortars
  bool has_v[kSizeClasses] = {false, false, false, false}, has_m[kSizeClasses] = {false, false, false, false};
  for (size_t b = 0; b < m->h_bucket_key.size(); ++b) {
    const auto& k = m->h_bucket_key[b];
    has_v[elem_size_class((k[0] + 1) * (k[1] + 1) * (k[2] + 1))] = true;
  }
  for (const auto& g : m->h_mgroups) has_m[mortar_size_class(std::max(g.la, g.ra) * std::max(g.lb, g.rb))] = true;
  double* r = nullptr;
  if ((e = cudaMalloc(&r, sizeof(double) * 5 * (size_t)m->n_nodes))) return status_of(e);
  dg_tiles rep;
  fill_budgets(m, &rep);
  dg_status st = DG_OK;
  // the face buffer the volume kernel lifts from, and the gradient (its values only need to be finite)
  if (m->phys.eqs == DG_NAVIER_STOKES) {
    if ((e = dgk::face_qhat(m, q)) || (e = dgk::gradient(m, q, m->d_grad, false))) st = status_of(e);
  }
  // coordinate descent: one class at a time, every candidate budget with the
  // others held, timed on the whole production launch; keep the fastest
  for (int pass = 0; pass < 2 && st == DG_OK; ++pass) {   // 0: volume tiles, 1: mortar batches
    int* budget = pass ? m->mortar_budget : m->vol_budget;
    const bool* has = pass ? has_m : has_v;
    double best = 0.0;
    st = rebuild(m);
    if (st == DG_OK && !pass) st = status_of(dgk::face_flux(m, q, m->d_grad, false));
    if (st == DG_OK) st = pass ? time_faces(m, q, reps, &best) : time_volume(m, q, r, reps, &best);
    for (int k = 0; k < kSizeClasses && st == DG_OK; ++k) {
      if (!has[k]) continue;
      (pass ? rep.mortar_ms_default : rep.vol_ms_default)[k] = best;
      const int keep = budget[k];
      int pick = keep;
      for (int c = 0; c < kNumCand && st == DG_OK; ++c) {
        if (kCandidates[c] == keep) continue;
        budget[k] = kCandidates[c];
        double t = 0.0;
        st = rebuild(m);
        if (st == DG_OK) st = pass ? time_faces(m, q, reps, &t) : time_volume(m, q, r, reps, &t);
        if (st == DG_OK && t < best) {
          best = t;
          pick = kCandidates[c];
        }
      }
      budget[k] = pick;
      (pass ? rep.mortar_ms : rep.vol_ms)[k] = best;
    }
  }
  cudaFree(r);
  if (st == DG_OK) st = rebuild(m);
  if (st != DG_OK) return st;
  std::copy(m->vol_budget, m->vol_budget + kSizeClasses, rep.vol_budget);
  std::copy(m->mortar_budget, m->mortar_budget + kSizeClasses, rep.mortar_budget);
  if (out) *out = rep;
  return DG_OK;
}
