// adapt.cu -- device support of the p-adaptation strategies (Sec. 2.4, 3.2):
// CFL-adaptive time integration to a given time, replayed as CUDA graphs
// (dg_advance), and the truncation-error extrapolation to N_i >= P_i
// (dg_tau_extrapolate).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <vector>

#include "dg.h"
#include "dg_internal.h"

namespace {

// device block of dg_advance
struct AdvState {
  double cfl, t_end, dt, steps;
};

// The clipped CFL step: dt = min(cfl / s_max, t_end - t).  The step that
// reaches t_end sets t = t_end exactly; once there, dt = 0 (an empty step).
__global__ void advance_clip_kernel(const unsigned long long* smax_bits, AdvState* a, double* t) {
  const double s = __longlong_as_double((long long)*smax_bits);
  double dt = a->cfl / s;
  const double tc = *t, rem = a->t_end - tc;
  if (!(rem > 0.0)) {
    dt = 0.0;
  } else if (dt >= rem) {
    dt = rem;
    *t = a->t_end;
  } else {
    *t = tc + dt;
  }
  a->dt = dt;
  if (dt > 0.0) a->steps += 1.0;
}

dg_status status_of(cudaError_t e) {
  return e == cudaSuccess ? DG_OK : e == cudaErrorMemoryAllocation ? DG_ERR_NOMEM : DG_ERR_CUDA;
}

// one step on m->stream: CFL reduction, clip, RK3 (three stages);
// trace_valid: the step before ran on the same q in this same sequence of
// launches, so its last stage left q's face traces in the mesh's buffer
dg_status advance_step(dg_mesh_impl* m, double* q, double* g, double* t, bool trace_valid) {
  unsigned long long* bits = reinterpret_cast<unsigned long long*>(m->d_scratch);
  AdvState* a = reinterpret_cast<AdvState*>(m->d_adv);
  cudaError_t e = dgk::max_dt_bits(m, q, bits);
  if (e) return status_of(e);
  dg_prof_begin(m, DG_KERNEL_MAX_DT, 1);
  advance_clip_kernel<<<1, 1, 0, m->stream>>>(bits, a, t);
  dg_prof_end(m, DG_KERNEL_MAX_DT);
  if ((e = cudaGetLastError())) return status_of(e);
  return rk_step_impl(m, q, g, &m->d_adv[2], trace_valid);
}

constexpr size_t kMaxGraphs = 24;

// n steps as one replay of a cached graph (captured on the first use)
dg_status advance_graph(dg_mesh_impl* m, double* q, double* g, double* t, int n) {
  dg_mesh_impl::AdvGraph* hit = nullptr;
  for (auto& c : m->adv_graphs)
    if (c.q == q && c.g == g && c.t == t && c.steps == n) hit = &c;
  if (!hit) {
    cudaError_t e;
    if (!m->cap_stream && (e = cudaStreamCreateWithFlags(&m->cap_stream, cudaStreamNonBlocking)))
      return status_of(e);
    if (m->adv_graphs.size() >= kMaxGraphs) {   // a bounded cache: start over
      for (auto& c : m->adv_graphs) cudaGraphExecDestroy(c.exec);
      m->adv_graphs.clear();
    }
    cudaStream_t saved = m->stream;
    const int64_t l0 = m->launches;
    if ((e = cudaStreamBeginCapture(m->cap_stream, cudaStreamCaptureModeThreadLocal))) return status_of(e);
    m->stream = m->cap_stream;
    dg_status st = DG_OK;
    for (int k = 0; k < n && st == DG_OK; ++k) st = advance_step(m, q, g, t, k > 0);   // a replay starts afresh
    m->stream = saved;
    cudaGraph_t graph = nullptr;
    e = cudaStreamEndCapture(m->cap_stream, &graph);
    const int64_t nl = m->launches - l0;
    m->launches = l0;
    if (st != DG_OK || e != cudaSuccess) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return st != DG_OK ? st : status_of(e);
    }
    cudaGraphExec_t exec = nullptr;
    e = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    if (e) return status_of(e);
    m->adv_graphs.push_back({q, g, t, n, exec, nl});
    hit = &m->adv_graphs.back();
  }
  cudaError_t e = cudaGraphLaunch(hit->exec, m->stream);
  if (e) return status_of(e);
  m->launches += hit->launches;
  return DG_OK;
}

dg_status run_steps(dg_mesh_impl* m, double* q, double* g, double* t, int64_t n, bool graphs) {
  bool traced = false;   // an eager step of this call ran before: q's face traces are in the buffer
  while (n > 0) {
    if (!graphs || !m->adv_warm) {
      dg_status st = advance_step(m, q, g, t, traced);
      if (st != DG_OK) return st;
      m->adv_warm = true;
      traced = true;
      --n;
      continue;
    }
    traced = false;
    int b = 32;
    while (b > n) b >>= 1;
    dg_status st = advance_graph(m, q, g, t, b);
    if (st != DG_OK) return st;
    n -= b;
  }
  return DG_OK;
}

// --------------------------------------------------------------------------
// Truncation-error extrapolation: one warp per element.
// --------------------------------------------------------------------------
struct ExtrapParams {
  int n_elem, n_sweep, n_target, n_fit;
  double tau_floor;
  int decoupled, accumulate;
  const int32_t* orders;          // [e][3]
  int32_t lut[DG_MAX_ORDER * DG_MAX_ORDER * DG_MAX_ORDER];   // (N1,N2,N3) -> first sweep index, or -1
  uint16_t tg[DG_MAX_ORDER * DG_MAX_ORDER * DG_MAX_ORDER];   // targets, (N1-1) | (N2-1) << 4 | (N3-1) << 8
};

__device__ __forceinline__ int lut_index(int a, int b, int c) {
  return (a - 1) + DG_MAX_ORDER * ((b - 1) + DG_MAX_ORDER * (c - 1));
}

template <typename T>
__global__ void extrap_kernel(const T* __restrict__ map, T* __restrict__ out, const __grid_constant__ ExtrapParams P) {
  const int lane = threadIdx.x & 31;
  const int e = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  if (e >= P.n_elem) return;
  const T* row = map + (int64_t)e * P.n_sweep;
  const int p0 = P.orders[3 * e], p1 = P.orders[3 * e + 1], p2 = P.orders[3 * e + 2];
  // lanes 0..2: the fit of direction lane; kind 0 exponential, 1 zero, 2 infinity
  int kind = 2;
  double fa = 0.0, fb = 0.0;
  if (lane < 3) {
    const int Pi = lane == 0 ? p0 : lane == 1 ? p1 : p2;
    auto dval = [&](int n) -> double {
      const int a = lane == 0 ? n : p0, b = lane == 1 ? n : p1, c = lane == 2 ? n : p2;
      const int s = P.lut[lut_index(a, b, c)];
      return s >= 0 ? (double)row[s] : -1.0;
    };
    if (Pi >= 2) {
      const double last = dval(Pi - 1);
      if (last >= 0.0 && last <= P.tau_floor) {
        kind = 1;
      } else {
        int lo = P.n_fit > 0 ? Pi - P.n_fit : 1;
        lo = lo < 1 ? 1 : lo;
        double sx = 0.0, sy = 0.0, sxx = 0.0, sxy = 0.0;
        int cnt = 0;
        for (int n = lo; n < Pi; ++n) {
          const double v = dval(n);
          if (!(v > 0.0)) continue;
          const double y = log(v);
          sx += n;
          sy += y;
          sxx += (double)n * n;
          sxy += n * y;
          ++cnt;
        }
        if (cnt >= 2) {
          const double xm = sx / cnt, ym = sy / cnt;
          const double slope = (sxy - cnt * xm * ym) / (sxx - cnt * xm * xm);
          if (slope < 0.0) {
            kind = 0;
            fb = slope;
            fa = ym - slope * xm;
          }
        }
      }
    }
  }
  int kd[3];
  double A[3], B[3];
  for (int i = 0; i < 3; ++i) {
    kd[i] = __shfl_sync(0xffffffffu, kind, i);
    A[i] = __shfl_sync(0xffffffffu, fa, i);
    B[i] = __shfl_sync(0xffffffffu, fb, i);
  }
  const int Pv[3] = {p0, p1, p2};
  T* orow = out + (int64_t)e * P.n_target;
  for (int t = lane; t < P.n_target; t += 32) {
    const int code = P.tg[t];
    const int N[3] = {(code & 15) + 1, ((code >> 4) & 15) + 1, ((code >> 8) & 15) + 1};
    double v;
    if (!P.decoupled) {
      int Nc[3];
      for (int i = 0; i < 3; ++i) Nc[i] = N[i] < Pv[i] ? N[i] : Pv[i];
      if (Nc[0] == p0 && Nc[1] == p1 && Nc[2] == p2) {
        v = 0.0;
      } else {
        const int s = P.lut[lut_index(Nc[0], Nc[1], Nc[2])];
        v = s >= 0 ? (double)row[s] : -1.0;
      }
      if (v >= 0.0)
        for (int i = 0; i < 3; ++i)
          if (N[i] >= Pv[i]) v += kd[i] == 0 ? exp(A[i] + B[i] * N[i]) : kd[i] == 1 ? 0.0 : (double)INFINITY;
    } else {
      v = 0.0;
      for (int i = 0; i < 3 && v >= 0.0; ++i) {
        double c;
        if (N[i] < Pv[i]) {
          int Nd[3] = {p0, p1, p2};
          Nd[i] = N[i];
          const int s = P.lut[lut_index(Nd[0], Nd[1], Nd[2])];
          c = s >= 0 ? (double)row[s] : -1.0;
        } else {
          c = kd[i] == 0 ? exp(A[i] + B[i] * N[i]) : kd[i] == 1 ? 0.0 : (double)INFINITY;
        }
        v = c < 0.0 ? -1.0 : v + c;
      }
    }
    const T tv = (T)v;
    orow[t] = P.accumulate ? (tv > orow[t] ? tv : orow[t]) : tv;
  }
}

}  // namespace

void dg_advance_release(dg_mesh_impl* m) {
  for (auto& c : m->adv_graphs) cudaGraphExecDestroy(c.exec);
  m->adv_graphs.clear();
  if (m->cap_stream) cudaStreamDestroy(m->cap_stream);
  m->cap_stream = nullptr;
  m->adv_warm = false;
}

extern "C" dg_status dg_advance(dg_mesh* mesh, double* q, double* g, double* t_dev, double t_end, double cfl,
                                int64_t max_steps, uint32_t flags, int64_t* steps_out) {
  dg_mesh_impl* m = mesh;
  if (!m || !q || !g || !t_dev || q == g || !(cfl > 0.0) || max_steps < 0 || std::isnan(t_end) ||
      (flags & ~DG_ADVANCE_EAGER))
    return DG_ERR_ARG;
  if (m->faces_unsupported) return DG_ERR_UNSUPPORTED;
  cudaError_t e;
  if (!m->d_adv && (e = cudaMalloc(&m->d_adv, sizeof(AdvState)))) return status_of(e);
  const AdvState init{cfl, t_end, 0.0, 0.0};
  if ((e = cudaMemcpyAsync(m->d_adv, &init, sizeof(init), cudaMemcpyHostToDevice, m->stream))) return status_of(e);
  const bool graphs = !(flags & DG_ADVANCE_EAGER) && !m->prof_on;
  dg_status st = DG_OK;
  if (std::isinf(t_end) && t_end > 0.0) {
    st = run_steps(m, q, g, t_dev, max_steps, graphs);
  } else {
    // batches sized from the last step: enough to reach t_end, in powers of two up to 32
    int64_t taken = 0, batch = 1;
    while (st == DG_OK && taken < max_steps) {
      const int64_t b = std::min(batch, max_steps - taken);
      st = run_steps(m, q, g, t_dev, b, graphs);
      if (st != DG_OK) break;
      taken += b;
      AdvState a;
      double t = 0.0;
      if ((e = cudaMemcpyAsync(&a, m->d_adv, sizeof(a), cudaMemcpyDeviceToHost, m->stream)) ||
          (e = cudaMemcpyAsync(&t, t_dev, sizeof(t), cudaMemcpyDeviceToHost, m->stream)) ||
          (e = cudaStreamSynchronize(m->stream))) {
        st = status_of(e);
        break;
      }
      if (!(t < t_end) || !(a.dt > 0.0)) break;
      const double need = std::ceil((t_end - t) / a.dt);
      batch = 1;
      while (batch < 32 && (double)batch < need) batch <<= 1;
    }
  }
  if (st == DG_OK && steps_out) {
    AdvState a;
    if ((e = cudaMemcpyAsync(&a, m->d_adv, sizeof(a), cudaMemcpyDeviceToHost, m->stream)) ||
        (e = cudaStreamSynchronize(m->stream)))
      return status_of(e);
    *steps_out = (int64_t)a.steps;
  }
  return st;
}

extern "C" dg_status dg_tau_extrapolate(dg_mesh* mesh, const void* map, int32_t map_fp32, const int32_t* sweep,
                                        int32_t n_sweep, const int32_t* targets, int32_t n_targets, int32_t n_fit,
                                        double tau_floor, uint32_t flags, void* map_out) {
  dg_mesh_impl* m = mesh;
  constexpr int kLut = DG_MAX_ORDER * DG_MAX_ORDER * DG_MAX_ORDER;
  if (!m || !map || !sweep || n_sweep <= 0 || !targets || n_targets <= 0 || n_targets > kLut || !map_out ||
      map == map_out || std::isnan(tau_floor) || (flags & ~(DG_EXTRAP_DECOUPLED | DG_EXTRAP_ACCUM_MAX)))
    return DG_ERR_ARG;
  for (int i = 0; i < 3 * n_sweep; ++i)
    if (sweep[i] < 1 || sweep[i] > DG_MAX_ORDER) return DG_ERR_ARG;
  for (int i = 0; i < 3 * n_targets; ++i)
    if (targets[i] < 1 || targets[i] > DG_MAX_ORDER) return DG_ERR_ARG;
  ExtrapParams P;
  P.n_elem = m->n_elem;
  P.n_sweep = n_sweep;
  P.n_target = n_targets;
  P.n_fit = n_fit;
  P.tau_floor = tau_floor;
  P.decoupled = (flags & DG_EXTRAP_DECOUPLED) != 0;
  P.accumulate = (flags & DG_EXTRAP_ACCUM_MAX) != 0;
  P.orders = m->d_ord;
  std::fill(P.lut, P.lut + kLut, -1);
  for (int s = n_sweep - 1; s >= 0; --s)   // the first occurrence wins
    P.lut[(sweep[3 * s] - 1) + DG_MAX_ORDER * ((sweep[3 * s + 1] - 1) + DG_MAX_ORDER * (sweep[3 * s + 2] - 1))] = s;
  for (int t = 0; t < n_targets; ++t)
    P.tg[t] = (uint16_t)((targets[3 * t] - 1) | (targets[3 * t + 1] - 1) << 4 | (targets[3 * t + 2] - 1) << 8);
  const int threads = 256;
  const int64_t grid = ((int64_t)m->n_elem * 32 + threads - 1) / threads;
  dg_prof_begin(m, DG_KERNEL_EXTRAP, 1);
  if (map_fp32)
    extrap_kernel<float><<<(unsigned)grid, threads, 0, m->stream>>>(static_cast<const float*>(map),
                                                                     static_cast<float*>(map_out), P);
  else
    extrap_kernel<double><<<(unsigned)grid, threads, 0, m->stream>>>(static_cast<const double*>(map),
                                                                      static_cast<double*>(map_out), P);
  dg_prof_end(m, DG_KERNEL_EXTRAP);
  return status_of(cudaGetLastError());
}
