// basis.cpp -- host construction of the 1D Gauss-Lobatto tables of libdg.
//
// Sec. 2.1: the DGSEM uses tensor-product Lagrange bases on the N+1
// Gauss-Lobatto (GL) nodes with the matching quadrature.  Here:
//   * GL nodes: Newton iteration on q(x) = L_{N+1}(x) - L_{N-1}(x), which
//     vanishes at all N+1 GL nodes (it is a multiple of (1-x^2) L_N'(x));
//   * weights w_j = 2 / (N(N+1) L_N(x_j)^2);
//   * derivative matrix from barycentric weights (Berrut & Trefethen 2004):
//     D_ij = (lam_j/lam_i)/(x_i - x_j), D_ii = -sum_{j!=i} D_ij;
//   * interpolation by the barycentric formula of the second kind, exact
//     identity where a target node coincides with a source node;
//   * L2 projection Pi = M^{-1} B, M the exact mass matrix of the target
//     basis (by the source GL rule, exact for degree 2*t <= 2*f-1) and
//     B_im = w_m ell_i(x_m); M^{-1} through a Cholesky factorisation.
#include <cmath>
#include <cstring>
#include <vector>

#include "dg_internal.h"

namespace dgb {

static void legendre_pair(int n, double x, double* Ln, double* Lnm1) {
  // L_n(x) and L_{n-1}(x) by Bonnet's recurrence
  double a = 1.0, b = x;  // L_0, L_1
  if (n == 0) { *Ln = 1.0; *Lnm1 = 0.0; return; }
  for (int k = 2; k <= n; ++k) {
    double c = ((2 * k - 1) * x * b - (k - 1) * a) / k;
    a = b;
    b = c;
  }
  *Ln = b;
  *Lnm1 = a;
}

void gl_nodes_weights(int N, double* x, double* w) {
  for (int j = 0; j <= N; ++j) {
    // initial guess: Chebyshev-Gauss-Lobatto point
    double t = -std::cos(M_PI * j / N);
    if (j == 0) { x[j] = -1.0; continue; }
    if (j == N) { x[j] = 1.0; continue; }
    for (int it = 0; it < 200; ++it) {
      // q = L_{N+1} - L_{N-1}; q' = (2N+1) L_N
      double LNp1, LN, LNm1, tmp;
      legendre_pair(N + 1, t, &LNp1, &LN);
      legendre_pair(N - 1, t, &LNm1, &tmp);
      double q = LNp1 - LNm1;
      double dq = (2.0 * N + 1.0) * LN;
      double step = q / dq;
      t -= step;
      if (std::fabs(step) <= 1e-17) break;
    }
    x[j] = t;
  }
  for (int j = 0; j < (N + 1) / 2; ++j) {  // symmetric pairs
    double s = 0.5 * (x[N - j] - x[j]);
    x[j] = -s;
    x[N - j] = s;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  for (int j = 0; j <= N; ++j) {
    double LN, LNm1;
    legendre_pair(N, x[j], &LN, &LNm1);
    w[j] = 2.0 / (N * (N + 1.0) * LN * LN);
  }
}

static void bary_weights(const double* x, int n, double* lam) {
  for (int j = 0; j < n; ++j) {
    double p = 1.0;
    for (int m = 0; m < n; ++m)
      if (m != j) p *= (x[j] - x[m]);
    lam[j] = 1.0 / p;
  }
}

void deriv_matrix(int N, double* D) {
  int n = N + 1;
  double x[DG_NP1], w[DG_NP1], lam[DG_NP1];
  gl_nodes_weights(N, x, w);
  bary_weights(x, n, lam);
  for (int i = 0; i < n; ++i) {
    double diag = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      double v = (lam[j] / lam[i]) / (x[i] - x[j]);
      D[i * n + j] = v;
      diag -= v;
    }
    D[i * n + i] = diag;
  }
}

void interp_matrix(const double* xf, int nf, const double* xt, int nt, double* I) {
  double lam[64];
  bary_weights(xf, nf, lam);
  for (int i = 0; i < nt; ++i) {
    int hit = -1;
    for (int j = 0; j < nf; ++j)
      if (xt[i] == xf[j]) hit = j;
    if (hit >= 0) {
      for (int j = 0; j < nf; ++j) I[i * nf + j] = (j == hit) ? 1.0 : 0.0;
      continue;
    }
    double den = 0.0;
    for (int j = 0; j < nf; ++j) den += lam[j] / (xt[i] - xf[j]);
    for (int j = 0; j < nf; ++j) I[i * nf + j] = (lam[j] / (xt[i] - xf[j])) / den;
  }
}

static void projection_matrix(int f, int t, double* Pm) {
  int nf = f + 1, nt = t + 1;
  double xf[DG_NP1], wf[DG_NP1], xt[DG_NP1], wt[DG_NP1];
  gl_nodes_weights(f, xf, wf);
  gl_nodes_weights(t, xt, wt);
  if (f == t) {
    for (int i = 0; i < nt; ++i)
      for (int m = 0; m < nf; ++m) Pm[i * nf + m] = (i == m) ? 1.0 : 0.0;
    return;
  }
  // Lt[m][i] = ell^t_i(xf_m)
  double Lt[DG_NP1 * DG_NP1];
  interp_matrix(xt, nt, xf, nf, Lt);
  double M[DG_NP1 * DG_NP1];
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < nt; ++j) {
      double s = 0.0;
      for (int m = 0; m < nf; ++m) s += wf[m] * Lt[m * nt + i] * Lt[m * nt + j];
      M[i * nt + j] = s;
    }
  // Cholesky M = C C^T (lower C, in place)
  double C[DG_NP1 * DG_NP1];
  std::memset(C, 0, sizeof(C));
  for (int j = 0; j < nt; ++j) {
    double s = M[j * nt + j];
    for (int k = 0; k < j; ++k) s -= C[j * nt + k] * C[j * nt + k];
    C[j * nt + j] = std::sqrt(s);
    for (int i = j + 1; i < nt; ++i) {
      double r = M[i * nt + j];
      for (int k = 0; k < j; ++k) r -= C[i * nt + k] * C[j * nt + k];
      C[i * nt + j] = r / C[j * nt + j];
    }
  }
  // solve M Pi = B column by column
  for (int m = 0; m < nf; ++m) {
    double y[DG_NP1];
    for (int i = 0; i < nt; ++i) {
      double r = wf[m] * Lt[m * nt + i];
      for (int k = 0; k < i; ++k) r -= C[i * nt + k] * y[k];
      y[i] = r / C[i * nt + i];
    }
    for (int i = nt - 1; i >= 0; --i) {
      double r = y[i];
      for (int k = i + 1; k < nt; ++k) r -= C[k * nt + i] * Pm[k * nf + m];
      Pm[i * nf + m] = r / C[i * nt + i];
    }
  }
}

void build_tables(BasisOffsets* off, std::vector<double>* data) {
  std::vector<double>& d = *data;
  d.clear();
  std::memset(off, 0, sizeof(*off));
  auto grab = [&](int n) {
    int o = (int)d.size();
    d.resize(d.size() + n);
    return o;
  };
  for (int N = 1; N <= DG_MAX_ORDER; ++N) {
    int n = N + 1;
    off->X[N] = grab(n);
    off->W[N] = grab(n);
    gl_nodes_weights(N, &d[off->X[N]], &d[off->W[N]]);
    off->D[N] = grab(n * n);
    deriv_matrix(N, &d[off->D[N]]);
  }
  for (int f = 1; f <= DG_MAX_ORDER; ++f)
    for (int t = 1; t <= DG_MAX_ORDER; ++t) {
      off->I[f][t] = grab((t + 1) * (f + 1));
      interp_matrix(&d[off->X[f]], f + 1, &d[off->X[t]], t + 1, &d[off->I[f][t]]);
      if (t <= f) {
        off->P[f][t] = grab((t + 1) * (f + 1));
        projection_matrix(f, t, &d[off->P[f][t]]);
      } else {
        off->P[f][t] = -1;
      }
    }
  off->total = (int)d.size();
}

}  // namespace dgb
