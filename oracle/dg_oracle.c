/*
 * dg_oracle.c -- plain FP64 CPU oracle for the DGSEM hot path of
 * Rueda-Ramirez, Ntoukas, Rubio, Valero, Ferrer, "Truncation Error-Based
 * Anisotropic p-Adaptation for Unsteady Flows for High-Order Discontinuous
 * Galerkin Methods" (arXiv 2210.03523).
 *
 * TEST INFRASTRUCTURE ONLY.  This file is the slow, obviously-correct
 * reference that the CUDA library is checked against.  Only the test suite,
 * the smoke check and the CPU-baseline leg of the benchmark may load it; the
 * product path never does.  It shares no code, table or header with the CUDA
 * library: it builds its own Gauss-Lobatto tables, metrics, fluxes and
 * projections from their definitions.
 *
 * What it computes (paper section / equation it follows):
 *   - DGSEM semi-discretisation, Sec. 2.1, Eq. (DGSEMsystem): tensor-product
 *     Lagrange basis on Gauss-Lobatto (GL) nodes with N+1 point quadrature, per
 *     direction orders (N1,N2,N3).  Written in the strong form, which for GL
 *     collocation is algebraically the weak form of Eq. (DGSEMsystem) by the
 *     summation-by-parts property of the GL derivative matrix.
 *   - R(Q) := dQ/dt = -(M^N)^{-1} F^N(Q), Eqs. (DGMassMatrixLeft/Right), with
 *     the diagonal mass matrix M = diag(J_j w_j).
 *   - Roe's approximate Riemann solver for the advective numerical flux and
 *     BR1 (Bassi-Rebay 1) for q-hat and the viscous numerical flux, Sec. 3.
 *   - Williamson's low-storage three-stage RK3, Sec. 3.
 *   - Truncation error, new (unscaled) form Eq. (TEtildedef) and traditional
 *     (mass-scaled) form Eq. (TEdef); isolated / non-isolated, end of Sec. 2.2.
 *   - Unsteady tau-estimation in its variational DG form, Sec. 2.3 item 1:
 *     I^N F(q) ~ I^N (M^P)^{-1} F^P(q^P) and I^N q ~ I^N q^P.
 *   - The infinity-norm truncation error map per element and anisotropic
 *     coarse order, Sec. 2.3 / 2.4.
 *
 * Readings where the paper is silent (each one is listed in the design notes):
 *   - restriction I^N = interpolation (the paper: "simply sampling");
 *   - p-nonconforming faces: mortar of order max(N_L, N_R) per tangential
 *     direction, interpolation up, exact L2 projection down;
 *   - curvilinear metrics in Kopriva's conservative curl form;
 *   - no entropy fix in Roe;
 *   - isolated tau uses the isolated residual in both terms unless the caller
 *     passes its own R^P.
 *
 * Pins (each part checked against something other than itself, in the
 * tests named test_oracle_*.py):
 *   - GL tables: closed forms up to N = 4, numpy's Legendre roots, row sums
 *     of D, the summation-by-parts identity (basis);
 *   - residual: free-stream preservation (affine, sheared, curved, O-grid,
 *     with mortars), polynomial exactness of the pulse family across mortars,
 *     equality with an independent scalar upwind DGSEM, discrete
 *     conservation, the curl-form metric identities (residual);
 *   - Roe and viscous fluxes: consistency, upwinding, rotation invariance,
 *     the contact-wave reduction, closed forms of shear and conduction
 *     (fluxes); BR1 exact for linear states, viscous heating of a shear
 *     flow on uniform and mixed orders, no mass flux through a wall (ns);
 *   - RK3 and the CFL step: order conditions, the Taylor polynomial of a
 *     linear operator, design-order convergence of the pulse, its centroid
 *     moving with the flow, closed forms and invariants of both CFL terms
 *     (time);
 *   - tau: zero at N = P, closed forms of both forms, vanishing above the
 *     state's degree, the exact truncation error of an analytic solution,
 *     the scaling with element size, non-isolated tau (tau);
 *   - order projection, selection (the paper's Table 1), extrapolation,
 *     drivers, wall force and the finite-difference adjoint (their files).
 *
 * Layout (the interface both implementations agree on): element e has
 * n_e = (N1+1)(N2+1)(N3+1) nodes; the state of element e starts at
 * 5 * sum_{e'<e} n_e' doubles and is stored [var][k][j][i] with i fastest.
 * Variables are (rho, rho u, rho v, rho w, rho E).
 */
#define _USE_MATH_DEFINES
#include <math.h>
#include <stdlib.h>
#include <string.h>
#include <stdio.h>

#define NV 5
#define NMAX 16
#ifndef M_PI
#define M_PI 3.14159265358979323846
#endif

/* ------------------------------------------------------------------------ */
/* 1. One-dimensional basis: Gauss-Lobatto nodes, weights, Lagrange values,  */
/*    derivative matrix.  (Sec. 2.1: "quadrature rule of N+1 points")        */
/* ------------------------------------------------------------------------ */

/* Legendre polynomial L_N(x) and its first derivative by the three-term
 * recurrence (k+1) L_{k+1} = (2k+1) x L_k - k L_{k-1}. */
static void legendre(int N, double x, double* L, double* dL) {
  double l0 = 1.0, l1 = x, d0 = 0.0, d1 = 1.0;
  if (N == 0) { *L = 1.0; *dL = 0.0; return; }
  for (int k = 1; k < N; ++k) {
    double l2 = ((2.0 * k + 1.0) * x * l1 - k * l0) / (k + 1.0);
    double d2 = d0 + (2.0 * k + 1.0) * l1;   /* L'_{k+1} = L'_{k-1} + (2k+1) L_k */
    l0 = l1; l1 = l2; d0 = d1; d1 = d2;
  }
  *L = l1; *dL = d1;
}

/* GL nodes: x_0=-1, x_N=+1 and the N-1 roots of L_N'(x).  Newton on L_N'
 * with L_N'' from Legendre's equation (1-x^2) L'' = 2x L' - N(N+1) L,
 * started from the Chebyshev-Gauss-Lobatto points.  Weights
 * w_j = 2 / (N (N+1) L_N(x_j)^2). */
void orc_gl(int N, double* x, double* w) {
  x[0] = -1.0; x[N] = 1.0;
  for (int j = 1; j < N; ++j) {
    double xi = -cos(M_PI * j / N);
    for (int it = 0; it < 100; ++it) {
      double L, dL;
      legendre(N, xi, &L, &dL);
      double d2L = (2.0 * xi * dL - N * (N + 1.0) * L) / (1.0 - xi * xi);
      double dx = dL / d2L;
      xi -= dx;
      if (fabs(dx) < 1e-16) break;
    }
    x[j] = xi;
  }
  /* enforce the exact symmetry of the node set */
  for (int j = 0; j <= N / 2; ++j) {
    double s = 0.5 * (x[N - j] - x[j]);
    x[j] = -s; x[N - j] = s;
  }
  if (N % 2 == 0) x[N / 2] = 0.0;
  for (int j = 0; j <= N; ++j) {
    double L, dL;
    legendre(N, x[j], &L, &dL);
    w[j] = 2.0 / (N * (N + 1.0) * L * L);
  }
}

/* Lagrange basis polynomial ell_j(t) on nodes x[0..n-1], product form. */
static double lagrange(const double* x, int n, int j, double t) {
  double v = 1.0;
  for (int m = 0; m < n; ++m)
    if (m != j) v *= (t - x[m]) / (x[j] - x[m]);
  return v;
}

/* Derivative ell_j'(t), written out from the product rule:
 * ell_j'(t) = sum_{k!=j} 1/(x_j-x_k) prod_{m!=j,k} (t-x_m)/(x_j-x_m). */
static double lagrange_deriv(const double* x, int n, int j, double t) {
  double s = 0.0;
  for (int k = 0; k < n; ++k) {
    if (k == j) continue;
    double p = 1.0 / (x[j] - x[k]);
    for (int m = 0; m < n; ++m)
      if (m != j && m != k) p *= (t - x[m]) / (x[j] - x[m]);
    s += p;
  }
  return s;
}

/* GL derivative matrix D_ij = ell_j'(x_i), row-major (N+1)x(N+1). */
void orc_dmat(int N, double* D) {
  double x[NMAX + 1], w[NMAX + 1];
  orc_gl(N, x, w);
  for (int i = 0; i <= N; ++i)
    for (int j = 0; j <= N; ++j) D[i * (N + 1) + j] = lagrange_deriv(x, N + 1, j, x[i]);
}

/* Interpolation matrix from order Nf GL nodes to order Nt GL nodes:
 * I[i][j] = ell^{Nf}_j(x^{Nt}_i), shape (Nt+1) x (Nf+1).  This is the
 * restriction / prolongation operator I^N of Eq. (TEderivation1) read as
 * interpolation (sampling of the degree-Nf polynomial). */
void orc_interp_mat(int Nf, int Nt, double* I) {
  double xf[NMAX + 1], wf[NMAX + 1], xt[NMAX + 1], wt[NMAX + 1];
  orc_gl(Nf, xf, wf);
  orc_gl(Nt, xt, wt);
  for (int i = 0; i <= Nt; ++i)
    for (int j = 0; j <= Nf; ++j) I[i * (Nf + 1) + j] = lagrange(xf, Nf + 1, j, xt[i]);
}

/* L2 projection from order Nf to order Nt <= Nf: Pi = M^{-1} B with the
 * mass matrix M_ij = sum_m w^{Nf}_m ell^{Nt}_i(x^{Nf}_m) ell^{Nt}_j(x^{Nf}_m)
 * and B_im = w^{Nf}_m ell^{Nt}_i(x^{Nf}_m).  For Nt < Nf the Nf-point GL rule
 * integrates both products exactly, so Pi is the exact L2 projection of the
 * degree-Nf interpolant onto degree Nt: it reproduces polynomials of degree
 * <= Nt and keeps the integral (discrete conservation).  For Nt == Nf it is
 * the identity.  Shape (Nt+1) x (Nf+1).  M is inverted by Gauss-Jordan
 * elimination with partial pivoting. */
void orc_proj_mat(int Nf, int Nt, double* Pm) {
  double xf[NMAX + 1], wf[NMAX + 1], xt[NMAX + 1], wt[NMAX + 1];
  orc_gl(Nf, xf, wf);
  orc_gl(Nt, xt, wt);
  int nt = Nt + 1, nf = Nf + 1;
  double L[(NMAX + 1) * (NMAX + 1)], M[(NMAX + 1) * (NMAX + 1)];
  for (int i = 0; i < nt; ++i)
    for (int m = 0; m < nf; ++m) L[i * nf + m] = lagrange(xt, nt, i, xf[m]);
  for (int i = 0; i < nt; ++i)
    for (int j = 0; j < nt; ++j) {
      double s = 0.0;
      for (int m = 0; m < nf; ++m) s += wf[m] * L[i * nf + m] * L[j * nf + m];
      M[i * nt + j] = s;
    }
  /* augmented system [M | B], reduced to [I | Pi] */
  for (int i = 0; i < nt; ++i)
    for (int m = 0; m < nf; ++m) Pm[i * nf + m] = wf[m] * L[i * nf + m];
  for (int c = 0; c < nt; ++c) {
    int piv = c;
    for (int r = c + 1; r < nt; ++r)
      if (fabs(M[r * nt + c]) > fabs(M[piv * nt + c])) piv = r;
    if (piv != c) {
      for (int k = 0; k < nt; ++k) { double t = M[c * nt + k]; M[c * nt + k] = M[piv * nt + k]; M[piv * nt + k] = t; }
      for (int k = 0; k < nf; ++k) { double t = Pm[c * nf + k]; Pm[c * nf + k] = Pm[piv * nf + k]; Pm[piv * nf + k] = t; }
    }
    double d = M[c * nt + c];
    for (int k = 0; k < nt; ++k) M[c * nt + k] /= d;
    for (int k = 0; k < nf; ++k) Pm[c * nf + k] /= d;
    for (int r = 0; r < nt; ++r) {
      if (r == c) continue;
      double f = M[r * nt + c];
      if (f == 0.0) continue;
      for (int k = 0; k < nt; ++k) M[r * nt + k] -= f * M[c * nt + k];
      for (int k = 0; k < nf; ++k) Pm[r * nf + k] -= f * Pm[c * nf + k];
    }
  }
  (void)wt;
}

/* ------------------------------------------------------------------------ */
/* 2. Tensor-product helpers                                                  */
/* ------------------------------------------------------------------------ */

/* Apply a (nt x nf) matrix A along direction dir of a 3D array with extents
 * ext[3] (ext[dir] == nf); the result has ext[dir] replaced by nt.
 * Index of (i,j,k) is i + ext0*(j + ext1*k). */
static void apply_dir(const double* A, int nt, int nf, int dir, const int ext[3], const double* in, double* out) {
  int eo[3] = {ext[0], ext[1], ext[2]};
  eo[dir] = nt;
  for (int k = 0; k < eo[2]; ++k)
    for (int j = 0; j < eo[1]; ++j)
      for (int i = 0; i < eo[0]; ++i) {
        int o[3] = {i, j, k};
        double s = 0.0;
        for (int m = 0; m < nf; ++m) {
          int p[3] = {i, j, k};
          p[dir] = m;
          s += A[o[dir] * nf + m] * in[p[0] + ext[0] * (p[1] + ext[1] * p[2])];
        }
        out[i + eo[0] * (j + eo[1] * k)] = s;
      }
}

/* Map a 3D array of orders Nf to orders Nt with one 1D matrix per direction
 * (mats[d] has shape (Nt[d]+1) x (Nf[d]+1)). */
static void apply_3d(double* const mats[3], const int Nf[3], const int Nt[3], const double* in, double* out) {
  int ext[3] = {Nf[0] + 1, Nf[1] + 1, Nf[2] + 1};
  int nmax = 1;
  for (int d = 0; d < 3; ++d) nmax *= (Nf[d] > Nt[d] ? Nf[d] : Nt[d]) + 1;
  double* a = malloc(sizeof(double) * nmax);
  double* b = malloc(sizeof(double) * nmax);
  memcpy(a, in, sizeof(double) * ext[0] * ext[1] * ext[2]);
  for (int d = 0; d < 3; ++d) {
    apply_dir(mats[d], Nt[d] + 1, Nf[d] + 1, d, ext, a, b);
    ext[d] = Nt[d] + 1;
    double* t = a; a = b; b = t;
  }
  memcpy(out, a, sizeof(double) * ext[0] * ext[1] * ext[2]);
  free(a); free(b);
}

/* ------------------------------------------------------------------------ */
/* 3. Mesh, geometry and metric terms                                         */
/* ------------------------------------------------------------------------ */

typedef struct {
  int eqs;           /* 0 Euler, 1 Navier-Stokes */
  double gamma, mu, Pr, Rgas;
  double qinf[NV];   /* free-stream state used by far-field boundaries */
} ophys;

typedef struct {
  int N[3], n;
  double *X[3];       /* node coordinates */
  double *Ja[3][3];   /* Ja[i][d]: d-th Cartesian component of J a^i */
  double *J;          /* Jacobian */
} egeo;

typedef struct {
  int n_elem, G;
  int* ord;          /* [e][3] */
  int* nbr;          /* [e][6] faces (-x1,+x1,-x2,+x2,-x3,+x3); <0: boundary tag */
  long* off;         /* node offset per element, off[n_elem] = total */
  double* geom;      /* [e][(G+1)^3][3] equispaced geometry nodes */
  ophys ph;
  egeo* geo;         /* per element geometry at its own orders */
} omesh;

static int nnodes(const int N[3]) { return (N[0] + 1) * (N[1] + 1) * (N[2] + 1); }

static void egeo_free(egeo* g) {
  for (int d = 0; d < 3; ++d) free(g->X[d]);
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) free(g->Ja[i][d]);
  free(g->J);
}

/* Geometry of element e interpolated to the GL nodes of orders N, and its
 * metric terms.  The geometry is the degree-G polynomial through the
 * equispaced geometry nodes.  J = det(dX/dxi).  J a^i in Kopriva's
 * conservative curl form, J a^i_n = - e_i . curl_xi( X_l grad_xi X_m ),
 * (n,m,l) cyclic, with every product interpolated at the GL nodes and
 * every derivative taken with the GL derivative matrix. */
static void elem_geometry(const omesh* m, int e, const int N[3], egeo* g) {
  int G = m->G, ng = G + 1;
  int n = nnodes(N);
  g->N[0] = N[0]; g->N[1] = N[1]; g->N[2] = N[2]; g->n = n;
  double xg[NMAX + 1];
  for (int a = 0; a <= G; ++a) xg[a] = -1.0 + 2.0 * a / G;
  double xs[3][NMAX + 1], ws[3][NMAX + 1], D[3][(NMAX + 1) * (NMAX + 1)];
  for (int d = 0; d < 3; ++d) { orc_gl(N[d], xs[d], ws[d]); orc_dmat(N[d], D[d]); }
  for (int d = 0; d < 3; ++d) g->X[d] = calloc(n, sizeof(double));
  const double* gn = m->geom + (size_t)e * ng * ng * ng * 3;
  for (int k = 0; k <= N[2]; ++k)
    for (int j = 0; j <= N[1]; ++j)
      for (int i = 0; i <= N[0]; ++i) {
        int id = i + (N[0] + 1) * (j + (N[1] + 1) * k);
        for (int c = 0; c <= G; ++c)
          for (int b = 0; b <= G; ++b)
            for (int a = 0; a <= G; ++a) {
              double l = lagrange(xg, ng, a, xs[0][i]) * lagrange(xg, ng, b, xs[1][j]) * lagrange(xg, ng, c, xs[2][k]);
              int gid = a + ng * (b + ng * c);
              for (int d = 0; d < 3; ++d) g->X[d][id] += l * gn[gid * 3 + d];
            }
      }
  int ext[3] = {N[0] + 1, N[1] + 1, N[2] + 1};
  /* dX[d][i] = dX_d / dxi_i at the nodes */
  double* dX[3][3];
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < 3; ++i) {
      dX[d][i] = malloc(sizeof(double) * n);
      apply_dir(D[i], N[i] + 1, N[i] + 1, i, ext, g->X[d], dX[d][i]);
    }
  g->J = malloc(sizeof(double) * n);
  for (int p = 0; p < n; ++p) {
    double a11 = dX[0][0][p], a12 = dX[0][1][p], a13 = dX[0][2][p];
    double a21 = dX[1][0][p], a22 = dX[1][1][p], a23 = dX[1][2][p];
    double a31 = dX[2][0][p], a32 = dX[2][1][p], a33 = dX[2][2][p];
    g->J[p] = a11 * (a22 * a33 - a23 * a32) - a12 * (a21 * a33 - a23 * a31) + a13 * (a21 * a32 - a22 * a31);
  }
  double* W[3];
  double* dW = malloc(sizeof(double) * n);
  for (int c = 0; c < 3; ++c) W[c] = malloc(sizeof(double) * n);
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) g->Ja[i][d] = calloc(n, sizeof(double));
  for (int nn = 0; nn < 3; ++nn) {
    int mm = (nn + 1) % 3, ll = (nn + 2) % 3;
    /* W_c = X_l dX_m/dxi_c */
    for (int c = 0; c < 3; ++c)
      for (int p = 0; p < n; ++p) W[c][p] = g->X[ll][p] * dX[mm][c][p];
    /* curl components: (curl W)_0 = d1 W2 - d2 W1, (curl W)_1 = d2 W0 - d0 W2,
     * (curl W)_2 = d0 W1 - d1 W0; J a^i_n = -(curl W)_i */
    for (int i = 0; i < 3; ++i) {
      int a = (i + 1) % 3, b = (i + 2) % 3;
      apply_dir(D[a], N[a] + 1, N[a] + 1, a, ext, W[b], dW);
      for (int p = 0; p < n; ++p) g->Ja[i][nn][p] -= dW[p];
      apply_dir(D[b], N[b] + 1, N[b] + 1, b, ext, W[a], dW);
      for (int p = 0; p < n; ++p) g->Ja[i][nn][p] += dW[p];
    }
  }
  for (int c = 0; c < 3; ++c) free(W[c]);
  free(dW);
  for (int d = 0; d < 3; ++d)
    for (int i = 0; i < 3; ++i) free(dX[d][i]);
}

void* orc_mesh_new(int n_elem, int G, const double* geom, const int* nbr, const int* ord, int eqs, double gamma,
                   double mu, double Pr, double Rgas, const double* qinf) {
  omesh* m = calloc(1, sizeof(omesh));
  m->n_elem = n_elem; m->G = G;
  int ng = G + 1;
  m->ord = malloc(sizeof(int) * 3 * n_elem); memcpy(m->ord, ord, sizeof(int) * 3 * n_elem);
  m->nbr = malloc(sizeof(int) * 6 * n_elem); memcpy(m->nbr, nbr, sizeof(int) * 6 * n_elem);
  m->geom = malloc(sizeof(double) * 3 * ng * ng * ng * n_elem);
  memcpy(m->geom, geom, sizeof(double) * 3 * ng * ng * ng * n_elem);
  m->off = malloc(sizeof(long) * (n_elem + 1));
  m->off[0] = 0;
  for (int e = 0; e < n_elem; ++e) m->off[e + 1] = m->off[e] + nnodes(m->ord + 3 * e);
  m->ph.eqs = eqs; m->ph.gamma = gamma; m->ph.mu = mu; m->ph.Pr = Pr; m->ph.Rgas = Rgas;
  for (int v = 0; v < NV; ++v) m->ph.qinf[v] = qinf ? qinf[v] : 0.0;
  m->geo = calloc(n_elem, sizeof(egeo));
#pragma omp parallel for schedule(guided)
  for (int e = 0; e < n_elem; ++e) elem_geometry(m, e, m->ord + 3 * e, &m->geo[e]);
  return m;
}

void orc_mesh_free(void* h) {
  omesh* m = h;
  for (int e = 0; e < m->n_elem; ++e) egeo_free(&m->geo[e]);
  free(m->geo); free(m->ord); free(m->nbr); free(m->geom); free(m->off); free(m);
}

long orc_n_nodes(void* h) { omesh* m = h; return m->off[m->n_elem]; }

/* coordinates [e][d][node], offset 3*off[e] */
void orc_node_coords(void* h, double* xyz) {
  omesh* m = h;
  for (int e = 0; e < m->n_elem; ++e)
    for (int d = 0; d < 3; ++d)
      memcpy(xyz + 3 * m->off[e] + d * m->geo[e].n, m->geo[e].X[d], sizeof(double) * m->geo[e].n);
}

/* metric terms of element e at its own orders: Ja [i][d][node], J [node] */
void orc_elem_metrics(void* h, int e, const int* N, double* X, double* Ja, double* J) {
  omesh* m = h;
  egeo g;
  elem_geometry(m, e, N, &g);
  for (int d = 0; d < 3; ++d) memcpy(X + d * g.n, g.X[d], sizeof(double) * g.n);
  for (int i = 0; i < 3; ++i)
    for (int d = 0; d < 3; ++d) memcpy(Ja + (i * 3 + d) * g.n, g.Ja[i][d], sizeof(double) * g.n);
  memcpy(J, g.J, sizeof(double) * g.n);
  egeo_free(&g);
}

/* ------------------------------------------------------------------------ */
/* 4. Physics: Euler flux, Roe flux, Navier-Stokes viscous flux              */
/*    (Sec. 2.1 first-order form; Sec. 3: Roe and BR1)                       */
/* ------------------------------------------------------------------------ */

static double pressure(double gamma, const double* q) {
  return (gamma - 1.0) * (q[4] - 0.5 * (q[1] * q[1] + q[2] * q[2] + q[3] * q[3]) / q[0]);
}

/* Cartesian advective (Euler) flux in direction d. */
static void euler_flux(double gamma, const double* q, int d, double* f) {
  double p = pressure(gamma, q);
  double ud = q[1 + d] / q[0];
  f[0] = q[1 + d];
  f[1] = q[1] * ud;
  f[2] = q[2] * ud;
  f[3] = q[3] * ud;
  f[1 + d] += p;
  f[4] = ud * (q[4] + p);
}

void orc_euler_flux(double gamma, const double* q, int d, double* f) { euler_flux(gamma, q, d, f); }

/* Roe's approximate Riemann solver for the flux through a face with unit
 * normal n from state qL (behind) to qR (ahead):
 *   f = 1/2 (f(qL).n + f(qR).n) - 1/2 sum_k |lambda_k| alpha_k r_k
 * with Roe-averaged velocity, enthalpy and sound speed (Roe 1981, in the
 * usual wave decomposition: two acoustic waves, the entropy wave and the
 * two shear waves).  No entropy fix. */
void orc_roe(double gamma, const double* qL, const double* qR, const double* n, double* f) {
  double rL = qL[0], rR = qR[0];
  double uL[3] = {qL[1] / rL, qL[2] / rL, qL[3] / rL};
  double uR[3] = {qR[1] / rR, qR[2] / rR, qR[3] / rR};
  double pL = pressure(gamma, qL), pR = pressure(gamma, qR);
  double HL = (qL[4] + pL) / rL, HR = (qR[4] + pR) / rR;
  double sL = sqrt(rL), sR = sqrt(rR);
  double rt = sL * sR;
  double ut[3], q2 = 0.0, utn = 0.0, dun = 0.0;
  for (int c = 0; c < 3; ++c) {
    ut[c] = (sL * uL[c] + sR * uR[c]) / (sL + sR);
    q2 += ut[c] * ut[c];
    utn += ut[c] * n[c];
    dun += (uR[c] - uL[c]) * n[c];
  }
  double Ht = (sL * HL + sR * HR) / (sL + sR);
  double c2 = (gamma - 1.0) * (Ht - 0.5 * q2);
  double ct = sqrt(c2);
  double dr = rR - rL, dp = pR - pL;
  double a1 = (dp - rt * ct * dun) / (2.0 * c2);
  double a5 = (dp + rt * ct * dun) / (2.0 * c2);
  double a2 = dr - dp / c2;
  double l1 = fabs(utn - ct), l2 = fabs(utn), l5 = fabs(utn + ct);
  double dut[3], utdut = 0.0;
  for (int c = 0; c < 3; ++c) {
    dut[c] = (uR[c] - uL[c]) - dun * n[c];
    utdut += ut[c] * dut[c];
  }
  double diss[NV];
  diss[0] = l1 * a1 + l5 * a5 + l2 * a2;
  for (int c = 0; c < 3; ++c)
    diss[1 + c] = l1 * a1 * (ut[c] - ct * n[c]) + l5 * a5 * (ut[c] + ct * n[c]) + l2 * (a2 * ut[c] + rt * dut[c]);
  diss[4] = l1 * a1 * (Ht - utn * ct) + l5 * a5 * (Ht + utn * ct) + l2 * (a2 * 0.5 * q2 + rt * utdut);
  double fL[NV] = {0}, fR[NV] = {0}, t[NV];
  for (int d = 0; d < 3; ++d) {
    euler_flux(gamma, qL, d, t);
    for (int v = 0; v < NV; ++v) fL[v] += t[v] * n[d];
    euler_flux(gamma, qR, d, t);
    for (int v = 0; v < NV; ++v) fR[v] += t[v] * n[d];
  }
  for (int v = 0; v < NV; ++v) f[v] = 0.5 * (fL[v] + fR[v]) - 0.5 * diss[v];
}

/* Navier-Stokes viscous flux in direction d for state q and gradient of the
 * conservative variables gq[v*3+c] = d q_v / d x_c.  Stokes hypothesis,
 * constant viscosity mu, Fourier heat flux with kappa = mu c_p / Pr,
 * c_p = gamma R / (gamma - 1), T = p / (rho R). */
static void visc_flux(const ophys* ph, const double* q, const double* gq, int d, double* f) {
  double g1 = ph->gamma - 1.0, rho = q[0];
  double u[3] = {q[1] / rho, q[2] / rho, q[3] / rho};
  double p = pressure(ph->gamma, q);
  double T = p / (rho * ph->Rgas);
  double du[3][3], dT[3];
  for (int c = 0; c < 3; ++c) {
    for (int i = 0; i < 3; ++i) du[i][c] = (gq[(1 + i) * 3 + c] - u[i] * gq[c]) / rho;
    double dp = g1 * (gq[4 * 3 + c] - (u[0] * gq[3 + c] + u[1] * gq[6 + c] + u[2] * gq[9 + c]) +
                      0.5 * (u[0] * u[0] + u[1] * u[1] + u[2] * u[2]) * gq[c]);
    dT[c] = (dp - ph->Rgas * T * gq[c]) / (rho * ph->Rgas);
  }
  double div = du[0][0] + du[1][1] + du[2][2];
  double kappa = ph->mu * ph->gamma * ph->Rgas / (g1 * ph->Pr);
  double tau[3];
  for (int i = 0; i < 3; ++i) tau[i] = ph->mu * (du[i][d] + du[d][i]) - (i == d ? 2.0 / 3.0 * ph->mu * div : 0.0);
  f[0] = 0.0;
  f[1] = tau[0]; f[2] = tau[1]; f[3] = tau[2];
  f[4] = u[0] * tau[0] + u[1] * tau[1] + u[2] * tau[2] + kappa * dT[d];
}

void orc_visc_flux(int eqs, double gamma, double mu, double Pr, double Rgas, const double* q, const double* gq, int d,
                   double* f) {
  ophys ph = {eqs, gamma, mu, Pr, Rgas, {0}};
  visc_flux(&ph, q, gq, d, f);
}

/* Boundary states.  tag -1: far field (free-stream ghost); tag -2: adiabatic
 * no-slip wall (ghost with reversed velocity). */
static void bc_ghost(const ophys* ph, int tag, const double* qi, double* qg) {
  if (tag == -2) {
    qg[0] = qi[0]; qg[1] = -qi[1]; qg[2] = -qi[2]; qg[3] = -qi[3]; qg[4] = qi[4];
  } else {
    for (int v = 0; v < NV; ++v) qg[v] = ph->qinf[v];
  }
}

/* BR1 trace q-hat on a boundary: free stream at the far field, the interior
 * state brought to rest (same density and internal energy) at the wall. */
static void bc_qhat(const ophys* ph, int tag, const double* qi, double* qh) {
  if (tag == -2) {
    qh[0] = qi[0]; qh[1] = 0.0; qh[2] = 0.0; qh[3] = 0.0;
    qh[4] = qi[4] - 0.5 * (qi[1] * qi[1] + qi[2] * qi[2] + qi[3] * qi[3]) / qi[0];
  } else {
    for (int v = 0; v < NV; ++v) qh[v] = ph->qinf[v];
  }
}

/* ------------------------------------------------------------------------ */
/* 5. Faces and mortars                                                       */
/* ------------------------------------------------------------------------ */

static void tangential(int dir, int* t0, int* t1) {
  *t0 = (dir == 0) ? 1 : 0;
  *t1 = (dir == 2) ? 1 : 2;
}

/* volume index of face node (a,b) on face f of an element of orders N */
static int face_vol_index(const int N[3], int f, int a, int b) {
  int dir = f / 2, side = f % 2, t0, t1;
  tangential(dir, &t0, &t1);
  int idx[3];
  idx[dir] = side ? N[dir] : 0;
  idx[t0] = a;
  idx[t1] = b;
  return idx[0] + (N[0] + 1) * (idx[1] + (N[1] + 1) * idx[2]);
}

/* gather nvar fields of stride n (field c at base + c*n) onto face f */
static void face_gather(const int N[3], int f, const double* base, int n, int nvar, double* out) {
  int dir = f / 2, t0, t1;
  tangential(dir, &t0, &t1);
  int na = N[t0] + 1, nb = N[t1] + 1;
  for (int c = 0; c < nvar; ++c)
    for (int b = 0; b < nb; ++b)
      for (int a = 0; a < na; ++a) out[c * na * nb + a + na * b] = base[c * n + face_vol_index(N, f, a, b)];
}

/* map nvar face fields from a (p0+1)x(p1+1) grid to (q0+1)x(q1+1) with the
 * 1D matrices A0 ((q0+1)x(p0+1)) and A1 ((q1+1)x(p1+1)) */
static void face_map(const double* A0, const double* A1, int p0, int p1, int q0, int q1, int nvar, const double* in,
                     double* out) {
  int ext[3] = {p0 + 1, p1 + 1, 1};
  double* tmp = malloc(sizeof(double) * (q0 + 1) * (p1 + 1));
  for (int c = 0; c < nvar; ++c) {
    apply_dir(A0, q0 + 1, p0 + 1, 0, ext, in + c * (p0 + 1) * (p1 + 1), tmp);
    int e2[3] = {q0 + 1, p1 + 1, 1};
    apply_dir(A1, q1 + 1, p1 + 1, 1, e2, tmp, out + c * (q0 + 1) * (q1 + 1));
  }
  free(tmp);
}

typedef struct {
  int M0, M1, nm;        /* mortar orders and node count */
  double *qo, *qn;       /* [NV][nm] own / neighbour states at mortar nodes */
  double *go, *gn;       /* [NV*3][nm] gradients (NS only) */
  double *Ja;            /* [3][nm] own J a^dir at mortar nodes */
  int N0o, N1o;          /* own tangential orders */
} mortar;

/* Build the mortar of face f of element e: interpolate both traces (and the
 * gradient traces for NS) to the mortar orders max(N_own, N_nbr) per
 * tangential direction, and the own J a^dir to the mortar nodes. */
static void mortar_build(const omesh* m, int e, int f, const double* q, const double* g, mortar* mo) {
  int dir = f / 2, t0, t1;
  tangential(dir, &t0, &t1);
  int nb = m->nbr[6 * e + f];
  const int* No = m->ord + 3 * e;
  const int* Nn = m->ord + 3 * nb;
  int fn = f ^ 1;
  int M0 = No[t0] > Nn[t0] ? No[t0] : Nn[t0];
  int M1 = No[t1] > Nn[t1] ? No[t1] : Nn[t1];
  mo->M0 = M0; mo->M1 = M1; mo->nm = (M0 + 1) * (M1 + 1);
  mo->N0o = No[t0]; mo->N1o = No[t1];
  int nfo = (No[t0] + 1) * (No[t1] + 1), nfn = (Nn[t0] + 1) * (Nn[t1] + 1);
  int no = nnodes(No), nn = nnodes(Nn);
  double Io0[(NMAX + 1) * (NMAX + 1)], Io1[(NMAX + 1) * (NMAX + 1)];
  double In0[(NMAX + 1) * (NMAX + 1)], In1[(NMAX + 1) * (NMAX + 1)];
  orc_interp_mat(No[t0], M0, Io0); orc_interp_mat(No[t1], M1, Io1);
  orc_interp_mat(Nn[t0], M0, In0); orc_interp_mat(Nn[t1], M1, In1);
  int nvq = (m->ph.eqs == 1) ? NV * 4 : NV;   /* q and, for NS, its gradient */
  double* to = malloc(sizeof(double) * nvq * nfo);
  double* tn = malloc(sizeof(double) * nvq * nfn);
  face_gather(No, f, q + NV * m->off[e], no, NV, to);
  face_gather(Nn, fn, q + NV * m->off[nb], nn, NV, tn);
  if (m->ph.eqs == 1) {
    /* gradient element layout [c][v][node]; store as [v*3+c] on the face */
    for (int v = 0; v < NV; ++v)
      for (int c = 0; c < 3; ++c) {
        face_gather(No, f, g + 3 * NV * m->off[e] + (c * NV + v) * no, no, 1, to + (NV + v * 3 + c) * nfo);
        face_gather(Nn, fn, g + 3 * NV * m->off[nb] + (c * NV + v) * nn, nn, 1, tn + (NV + v * 3 + c) * nfn);
      }
  }
  double* mo_o = malloc(sizeof(double) * nvq * mo->nm);
  double* mo_n = malloc(sizeof(double) * nvq * mo->nm);
  face_map(Io0, Io1, No[t0], No[t1], M0, M1, nvq, to, mo_o);
  face_map(In0, In1, Nn[t0], Nn[t1], M0, M1, nvq, tn, mo_n);
  mo->qo = mo_o; mo->qn = mo_n;
  mo->go = (m->ph.eqs == 1) ? mo_o + NV * mo->nm : NULL;
  mo->gn = (m->ph.eqs == 1) ? mo_n + NV * mo->nm : NULL;
  double* jt = malloc(sizeof(double) * 3 * nfo);
  const egeo* ge = &m->geo[e];
  for (int c = 0; c < 3; ++c) face_gather(No, f, ge->Ja[dir][c], no, 1, jt + c * nfo);
  mo->Ja = malloc(sizeof(double) * 3 * mo->nm);
  face_map(Io0, Io1, No[t0], No[t1], M0, M1, 3, jt, mo->Ja);
  free(to); free(tn); free(jt);
}

static void mortar_free(mortar* mo) { free(mo->qo); free(mo->qn); free(mo->Ja); }

/* project nvar mortar fields back to the own face grid */
static void mortar_project(const mortar* mo, int nvar, const double* in, double* out) {
  double P0[(NMAX + 1) * (NMAX + 1)], P1[(NMAX + 1) * (NMAX + 1)];
  orc_proj_mat(mo->M0, mo->N0o, P0);
  orc_proj_mat(mo->M1, mo->N1o, P1);
  face_map(P0, P1, mo->M0, mo->M1, mo->N0o, mo->N1o, nvar, in, out);
}

/* point value of q and its gradient from a [var][node] face array */
static void pick(const double* a, int nvar, int np, int p, double* out) {
  for (int c = 0; c < nvar; ++c) out[c] = a[c * np + p];
}

/* Contravariant numerical flux F* in the +xi_dir direction at the own nodes
 * of face f of element e: |J a^dir| (Roe(q-, q+, n) - viscous numerical
 * flux . n), n = J a^dir / |J a^dir|, where q- is the state on the -xi_dir
 * side of the face.  Output Fs[v][face node]. */
static void face_flux(const omesh* m, int e, int f, const double* q, const double* g, double* Fs) {
  const ophys* ph = &m->ph;
  int dir = f / 2, side = f % 2, t0, t1;
  tangential(dir, &t0, &t1);
  const int* No = m->ord + 3 * e;
  int nf = (No[t0] + 1) * (No[t1] + 1), no = nnodes(No);
  int tag = m->nbr[6 * e + f];
  int ns = ph->eqs == 1;
  if (tag < 0) {
    double* tq = malloc(sizeof(double) * NV * nf);
    double* tg = malloc(sizeof(double) * NV * 3 * nf);
    double* tj = malloc(sizeof(double) * 3 * nf);
    face_gather(No, f, q + NV * m->off[e], no, NV, tq);
    if (ns)
      for (int v = 0; v < NV; ++v)
        for (int c = 0; c < 3; ++c)
          face_gather(No, f, g + 3 * NV * m->off[e] + (c * NV + v) * no, no, 1, tg + (v * 3 + c) * nf);
    for (int c = 0; c < 3; ++c) face_gather(No, f, m->geo[e].Ja[dir][c], no, 1, tj + c * nf);
    for (int p = 0; p < nf; ++p) {
      double qi[NV], qg[NV], ja[3], gi[NV * 3], fl[NV];
      pick(tq, NV, nf, p, qi);
      pick(tj, 3, nf, p, ja);
      bc_ghost(ph, tag, qi, qg);
      double area = sqrt(ja[0] * ja[0] + ja[1] * ja[1] + ja[2] * ja[2]);
      double nrm[3] = {ja[0] / area, ja[1] / area, ja[2] / area};
      if (side) orc_roe(ph->gamma, qi, qg, nrm, fl);
      else orc_roe(ph->gamma, qg, qi, nrm, fl);
      for (int v = 0; v < NV; ++v) fl[v] *= area;
      if (ns) {
        pick(tg, NV * 3, nf, p, gi);
        double fv[NV], fvn[NV] = {0};
        for (int d = 0; d < 3; ++d) {
          visc_flux(ph, qi, gi, d, fv);
          for (int v = 0; v < NV; ++v) fvn[v] += fv[v] * ja[d];
        }
        if (tag == -2) { fvn[0] = 0.0; fvn[4] = 0.0; }  /* no mass flux; adiabatic, resting wall */
        for (int v = 0; v < NV; ++v) fl[v] -= fvn[v];
      }
      for (int v = 0; v < NV; ++v) Fs[v * nf + p] = fl[v];
    }
    free(tq); free(tg); free(tj);
    return;
  }
  mortar mo;
  mortar_build(m, e, f, q, g, &mo);
  double* Fm = malloc(sizeof(double) * NV * mo.nm);
  for (int p = 0; p < mo.nm; ++p) {
    double qo[NV], qn[NV], ja[3], fl[NV];
    pick(mo.qo, NV, mo.nm, p, qo);
    pick(mo.qn, NV, mo.nm, p, qn);
    pick(mo.Ja, 3, mo.nm, p, ja);
    double area = sqrt(ja[0] * ja[0] + ja[1] * ja[1] + ja[2] * ja[2]);
    double nrm[3] = {ja[0] / area, ja[1] / area, ja[2] / area};
    if (side) orc_roe(ph->gamma, qo, qn, nrm, fl);
    else orc_roe(ph->gamma, qn, qo, nrm, fl);
    for (int v = 0; v < NV; ++v) fl[v] *= area;
    if (ns) {
      double go[NV * 3], gn[NV * 3], fa[NV], fb[NV];
      pick(mo.go, NV * 3, mo.nm, p, go);
      pick(mo.gn, NV * 3, mo.nm, p, gn);
      for (int d = 0; d < 3; ++d) {
        visc_flux(ph, qo, go, d, fa);
        visc_flux(ph, qn, gn, d, fb);
        for (int v = 0; v < NV; ++v) fl[v] -= 0.5 * (fa[v] + fb[v]) * ja[d];   /* BR1: average */
      }
    }
    for (int v = 0; v < NV; ++v) Fm[v * mo.nm + p] = fl[v];
  }
  mortar_project(&mo, NV, Fm, Fs);
  free(Fm);
  mortar_free(&mo);
}

/* BR1 surface quantity for the gradient equation, Eq. (DGSEMsystem:2):
 * S[v*3+c][face node] = q-hat_v (J a^dir)_c at the own face nodes, with
 * q-hat the average of both traces (projected from the mortar). */
static void face_qhat(const omesh* m, int e, int f, const double* q, double* S) {
  const ophys* ph = &m->ph;
  int dir = f / 2, t0, t1;
  tangential(dir, &t0, &t1);
  const int* No = m->ord + 3 * e;
  int nf = (No[t0] + 1) * (No[t1] + 1), no = nnodes(No);
  int tag = m->nbr[6 * e + f];
  if (tag < 0) {
    double* tq = malloc(sizeof(double) * NV * nf);
    double* tj = malloc(sizeof(double) * 3 * nf);
    face_gather(No, f, q + NV * m->off[e], no, NV, tq);
    for (int c = 0; c < 3; ++c) face_gather(No, f, m->geo[e].Ja[dir][c], no, 1, tj + c * nf);
    for (int p = 0; p < nf; ++p) {
      double qi[NV], qh[NV], ja[3];
      pick(tq, NV, nf, p, qi);
      pick(tj, 3, nf, p, ja);
      bc_qhat(ph, tag, qi, qh);
      for (int v = 0; v < NV; ++v)
        for (int c = 0; c < 3; ++c) S[(v * 3 + c) * nf + p] = qh[v] * ja[c];
    }
    free(tq); free(tj);
    return;
  }
  /* the mortar of the gradient pass needs no gradients: build it as Euler */
  omesh tmp = *m;
  tmp.ph.eqs = 0;
  mortar mo;
  mortar_build(&tmp, e, f, q, NULL, &mo);
  double* Sm = malloc(sizeof(double) * NV * 3 * mo.nm);
  for (int p = 0; p < mo.nm; ++p)
    for (int v = 0; v < NV; ++v) {
      double qh = 0.5 * (mo.qo[v * mo.nm + p] + mo.qn[v * mo.nm + p]);
      for (int c = 0; c < 3; ++c) Sm[(v * 3 + c) * mo.nm + p] = qh * mo.Ja[c * mo.nm + p];
    }
  mortar_project(&mo, NV * 3, Sm, S);
  free(Sm);
  mortar_free(&mo);
}

/* ------------------------------------------------------------------------ */
/* 6. Element operators                                                       */
/* ------------------------------------------------------------------------ */

/* Volume part of the BR1 gradient: J g_c = sum_i D^(i) (J a^i_c q).
 * Output Jg[c][v][node]. */
static void grad_volume(const egeo* geo, const double* qe, double* Jg) {
  const int* N = geo->N;
  int n = geo->n, ext[3] = {N[0] + 1, N[1] + 1, N[2] + 1};
  double D[3][(NMAX + 1) * (NMAX + 1)];
  for (int d = 0; d < 3; ++d) orc_dmat(N[d], D[d]);
  double* t = malloc(sizeof(double) * n);
  double* dt = malloc(sizeof(double) * n);
  memset(Jg, 0, sizeof(double) * 3 * NV * n);
  for (int c = 0; c < 3; ++c)
    for (int v = 0; v < NV; ++v)
      for (int i = 0; i < 3; ++i) {
        for (int p = 0; p < n; ++p) t[p] = geo->Ja[i][c][p] * qe[v * n + p];
        apply_dir(D[i], N[i] + 1, N[i] + 1, i, ext, t, dt);
        for (int p = 0; p < n; ++p) Jg[(c * NV + v) * n + p] += dt[p];
      }
  free(t); free(dt);
}

/* Volume part of the residual: vol[v] = sum_i D^(i) Ft^i_v with the
 * contravariant flux Ft^i = sum_d J a^i_d (f^a_d - f^nu_d); Ft is returned
 * too ([i][v][node]) for the surface terms.  ge (gradient [c][v][node]) is
 * used for Navier-Stokes only. */
static void residual_volume(const ophys* ph, const egeo* geo, const double* qe, const double* ge, double* vol,
                            double* Ft) {
  const int* N = geo->N;
  int n = geo->n, ext[3] = {N[0] + 1, N[1] + 1, N[2] + 1};
  double D[3][(NMAX + 1) * (NMAX + 1)];
  for (int d = 0; d < 3; ++d) orc_dmat(N[d], D[d]);
  memset(Ft, 0, sizeof(double) * 3 * NV * n);
  for (int p = 0; p < n; ++p) {
    double qp[NV], gp[NV * 3], f[NV], fv[NV];
    for (int v = 0; v < NV; ++v) qp[v] = qe[v * n + p];
    if (ph->eqs == 1)
      for (int v = 0; v < NV; ++v)
        for (int c = 0; c < 3; ++c) gp[v * 3 + c] = ge[(c * NV + v) * n + p];
    for (int d = 0; d < 3; ++d) {
      euler_flux(ph->gamma, qp, d, f);
      if (ph->eqs == 1) {
        visc_flux(ph, qp, gp, d, fv);
        for (int v = 0; v < NV; ++v) f[v] -= fv[v];
      }
      for (int i = 0; i < 3; ++i)
        for (int v = 0; v < NV; ++v) Ft[(i * NV + v) * n + p] += geo->Ja[i][d][p] * f[v];
    }
  }
  double* dt = malloc(sizeof(double) * n);
  memset(vol, 0, sizeof(double) * NV * n);
  for (int v = 0; v < NV; ++v)
    for (int i = 0; i < 3; ++i) {
      apply_dir(D[i], N[i] + 1, N[i] + 1, i, ext, Ft + (i * NV + v) * n, dt);
      for (int p = 0; p < n; ++p) vol[v * n + p] += dt[p];
    }
  free(dt);
}

/* Element-local (isolated) residual at the geometry geo: surface numerical
 * fluxes replaced by the inner flux (end of Sec. 2.2), so only the volume
 * term survives; for Navier-Stokes the BR1 gradient is element-local too. */
static void isolated_residual(const ophys* ph, const egeo* geo, const double* qe, double* re) {
  int n = geo->n;
  double* ge = NULL;
  if (ph->eqs == 1) {
    ge = malloc(sizeof(double) * 3 * NV * n);
    grad_volume(geo, qe, ge);
    for (int c = 0; c < 3; ++c)
      for (int v = 0; v < NV; ++v)
        for (int p = 0; p < n; ++p) ge[(c * NV + v) * n + p] /= geo->J[p];
  }
  double* Ft = malloc(sizeof(double) * 3 * NV * n);
  double* vol = malloc(sizeof(double) * NV * n);
  residual_volume(ph, geo, qe, ge, vol, Ft);
  for (int v = 0; v < NV; ++v)
    for (int p = 0; p < n; ++p) re[v * n + p] = -vol[v * n + p] / geo->J[p];
  free(Ft); free(vol); free(ge);
}

/* ------------------------------------------------------------------------ */
/* 7. Mesh-level operators                                                    */
/* ------------------------------------------------------------------------ */

/* BR1 gradient g = grad q of Eq. (DGSEMsystem:2), strong form:
 * J g_c = sum_i D^(i)(J a^i_c q) + sum over faces of the lifted
 * (q-hat - q) J a^i_c, +1/w_N on +xi faces and -1/w_0 on -xi faces.
 * Output layout [e][c][v][node] at offset 3*NV*off[e]. */
void orc_gradient(void* h, const double* q, double* g, int isolated) {
  omesh* m = h;
#pragma omp parallel for schedule(guided)
  for (int e = 0; e < m->n_elem; ++e) {
    const egeo* geo = &m->geo[e];
    const int* N = geo->N;
    int n = geo->n;
    double* Jg = g + 3 * NV * m->off[e];
    grad_volume(geo, q + NV * m->off[e], Jg);
    if (!isolated) {
      const double* qe = q + NV * m->off[e];
      for (int f = 0; f < 6; ++f) {
        int dir = f / 2, side = f % 2, t0, t1;
        tangential(dir, &t0, &t1);
        int na = N[t0] + 1, nb = N[t1] + 1, nf = na * nb;
        double* S = malloc(sizeof(double) * NV * 3 * nf);
        face_qhat(m, e, f, q, S);
        double x[NMAX + 1], w[NMAX + 1];
        orc_gl(N[dir], x, w);
        double wend = side ? w[N[dir]] : w[0];
        double sgn = side ? 1.0 : -1.0;
        for (int b = 0; b < nb; ++b)
          for (int a = 0; a < na; ++a) {
            int p = a + na * b, vi = face_vol_index(N, f, a, b);
            for (int v = 0; v < NV; ++v)
              for (int c = 0; c < 3; ++c) {
                double own = qe[v * n + vi] * geo->Ja[dir][c][vi];
                Jg[(c * NV + v) * n + vi] += sgn * (S[(v * 3 + c) * nf + p] - own) / wend;
              }
          }
        free(S);
      }
    }
    for (int c = 0; c < 3; ++c)
      for (int v = 0; v < NV; ++v)
        for (int p = 0; p < n; ++p) Jg[(c * NV + v) * n + p] /= geo->J[p];
  }
}

/* Residual R(Q) = dQ/dt = -(M^N)^{-1} F^N(Q), Eq. (DGMassMatrixRight), in
 * strong form: J R = -[ sum_i D^(i) Ft^i + lifted surface terms ], with the
 * lift (F* - Ft)/w_N on +xi faces and -(F* - Ft)/w_0 on -xi faces.
 * isolated != 0 gives the isolated residual (inner flux on every face). */
void orc_residual(void* h, const double* q, double* r, int isolated) {
  omesh* m = h;
  const ophys* ph = &m->ph;
  double* g = NULL;
  if (ph->eqs == 1) {
    g = malloc(sizeof(double) * 3 * NV * m->off[m->n_elem]);
    orc_gradient(h, q, g, isolated);
  }
#pragma omp parallel for schedule(guided)
  for (int e = 0; e < m->n_elem; ++e) {
    const egeo* geo = &m->geo[e];
    const int* N = geo->N;
    int n = geo->n;
    const double* qe = q + NV * m->off[e];
    const double* ge = g ? g + 3 * NV * m->off[e] : NULL;
    double* Ft = malloc(sizeof(double) * 3 * NV * n);
    double* vol = malloc(sizeof(double) * NV * n);
    residual_volume(ph, geo, qe, ge, vol, Ft);
    if (!isolated) {
      for (int f = 0; f < 6; ++f) {
        int dir = f / 2, side = f % 2, t0, t1;
        tangential(dir, &t0, &t1);
        int na = N[t0] + 1, nb = N[t1] + 1, nf = na * nb;
        double* Fs = malloc(sizeof(double) * NV * nf);
        face_flux(m, e, f, q, g, Fs);
        double x[NMAX + 1], w[NMAX + 1];
        orc_gl(N[dir], x, w);
        double wend = side ? w[N[dir]] : w[0];
        double sgn = side ? 1.0 : -1.0;
        for (int b = 0; b < nb; ++b)
          for (int a = 0; a < na; ++a) {
            int p = a + na * b, vi = face_vol_index(N, f, a, b);
            for (int v = 0; v < NV; ++v) vol[v * n + vi] += sgn * (Fs[v * nf + p] - Ft[(dir * NV + v) * n + vi]) / wend;
          }
        free(Fs);
      }
    }
    double* re = r + NV * m->off[e];
    for (int v = 0; v < NV; ++v)
      for (int p = 0; p < n; ++p) re[v * n + p] = -vol[v * n + p] / geo->J[p];
    free(Ft); free(vol);
  }
  free(g);
}

/* Williamson's low-storage RK3 (Sec. 3), three stages k = 1..3:
 *   G <- A_k G + dt R(Q),  Q <- Q + B_k G,
 * A = (0, -5/9, -153/128), B = (1/3, 15/16, 8/15). */
static const double RK_A[3] = {0.0, -5.0 / 9.0, -153.0 / 128.0};
static const double RK_B[3] = {1.0 / 3.0, 15.0 / 16.0, 8.0 / 15.0};

void orc_rk_coeffs(double* A, double* B) {
  for (int k = 0; k < 3; ++k) { A[k] = RK_A[k]; B[k] = RK_B[k]; }
}

void orc_rk_step(void* h, double* q, double* G, double dt) {
  omesh* m = h;
  long ns = NV * m->off[m->n_elem];
  double* r = malloc(sizeof(double) * ns);
  for (int k = 0; k < 3; ++k) {
    orc_residual(h, q, r, 0);
    for (long i = 0; i < ns; ++i) {
      G[i] = RK_A[k] * G[i] + dt * r[i];
      q[i] += RK_B[k] * G[i];
    }
  }
  free(r);
}

/* CFL time step (the paper defers the formula to HORSES3D; this is the
 * reading used throughout): dt = CFL / max over nodes of max(s_a, s_v),
 *   s_a = sum_i (N_i+1)^2 (|J a^i . v| + c |J a^i|) / (2 J),
 *   s_v = sum_i (N_i+1)^4 |J a^i|^2 / (4 J^2) * max(1, gamma/Pr) mu / rho  (NS). */
double orc_max_dt(void* h, const double* q, double cfl) {
  omesh* m = h;
  const ophys* ph = &m->ph;
  double smax = 0.0;
  for (int e = 0; e < m->n_elem; ++e) {
    const egeo* geo = &m->geo[e];
    int n = geo->n;
    const double* qe = q + NV * m->off[e];
    for (int p = 0; p < n; ++p) {
      double qp[NV];
      for (int v = 0; v < NV; ++v) qp[v] = qe[v * n + p];
      double rho = qp[0], u[3] = {qp[1] / rho, qp[2] / rho, qp[3] / rho};
      double c = sqrt(ph->gamma * pressure(ph->gamma, qp) / rho);
      double J = geo->J[p], sa = 0.0, sv = 0.0;
      for (int i = 0; i < 3; ++i) {
        double ja[3] = {geo->Ja[i][0][p], geo->Ja[i][1][p], geo->Ja[i][2][p]};
        double a2 = ja[0] * ja[0] + ja[1] * ja[1] + ja[2] * ja[2];
        double un = fabs(ja[0] * u[0] + ja[1] * u[1] + ja[2] * u[2]);
        double k2 = (geo->N[i] + 1.0) * (geo->N[i] + 1.0);
        sa += k2 * (un + c * sqrt(a2)) / (2.0 * J);
        sv += k2 * k2 * a2 / (4.0 * J * J);
      }
      double s = sa;
      if (ph->eqs == 1) {
        double nu = ph->mu / rho * (ph->gamma / ph->Pr > 1.0 ? ph->gamma / ph->Pr : 1.0);
        if (sv * nu > s) s = sv * nu;
      }
      if (s > smax) smax = s;
    }
  }
  return cfl / smax;
}

/* Time integration to a given time (Sec. 3.1: the time-step size follows
 * the CFL condition at every step).  Steps of size orc_max_dt from *t; the
 * step that would pass t_end is shortened to land on it exactly.  At most
 * max_steps steps; returns the number taken and leaves *t at the new time. */
int orc_advance(void* h, double* q, double* G, double cfl, double* t, double t_end, int max_steps) {
  int n = 0;
  while (n < max_steps && *t < t_end) {
    double dt = orc_max_dt(h, q, cfl);
    const double rem = t_end - *t;
    const int last = dt >= rem;
    if (last) dt = rem;
    orc_rk_step(h, q, G, dt);
    *t = last ? t_end : *t + dt;
    ++n;
  }
  return n;
}

/* ------------------------------------------------------------------------ */
/* 8. Truncation-error estimation (Sec. 2.2, 2.3)                             */
/* ------------------------------------------------------------------------ */

static void interp_elem(const int Nf[3], const int Nt[3], int nvar, const double* in, double* out) {
  double* mats[3];
  for (int d = 0; d < 3; ++d) {
    mats[d] = malloc(sizeof(double) * (Nt[d] + 1) * (Nf[d] + 1));
    orc_interp_mat(Nf[d], Nt[d], mats[d]);
  }
  int nf = nnodes(Nf), nt = nnodes(Nt);
  for (int c = 0; c < nvar; ++c) apply_3d(mats, Nf, Nt, in + c * nf, out + c * nt);
  for (int d = 0; d < 3; ++d) free(mats[d]);
}

/* infinity norms of the new form (Eq. TEtildedef) and the traditional form
 * tau = M tau-tilde = J_j w_j tau-tilde_j (Eq. TEdef) over all nodes and all
 * five variables; tt is tau-tilde at order N on geometry geo */
static void tau_norms(const egeo* geo, const double* tt, double* nnew, double* ntrad) {
  const int* N = geo->N;
  double x[3][NMAX + 1], w[3][NMAX + 1];
  for (int d = 0; d < 3; ++d) orc_gl(N[d], x[d], w[d]);
  double a = 0.0, b = 0.0;
  int n = geo->n;
  for (int v = 0; v < NV; ++v)
    for (int k = 0; k <= N[2]; ++k)
      for (int j = 0; j <= N[1]; ++j)
        for (int i = 0; i <= N[0]; ++i) {
          int p = i + (N[0] + 1) * (j + (N[1] + 1) * k);
          double t = tt[v * n + p];
          double s = geo->J[p] * w[0][i] * w[1][j] * w[2][k] * t;
          if (fabs(t) > a) a = fabs(t);
          if (fabs(s) > b) b = fabs(s);
        }
  *nnew = a; *ntrad = b;
}

static void store(double* out, int accumulate, double v) {
  if (accumulate) { if (v > *out) *out = v; }
  else *out = v;
}

/* Unsteady tau-estimation, variational DG form (Sec. 2.3 item 1):
 *   tau-tilde^N = I^N R^P(q^P) - R^N(I^N q^P)
 *              = (M^N)^{-1} F^N(I^N q^P) - I^N (M^P)^{-1} F^P(q^P),
 * the estimate of Eq. (TEtildedef); tau^N = M^N tau-tilde^N, Eq. (TEdef).
 * For every element e and sweep entry s (orders N_s): if N_s <= P_e
 * componentwise, out[e*ns+s] = max over nodes and variables of |tau|;
 * otherwise -1 (not estimable from the order P_e solution).
 * isolated != 0: R^N and (unless rP is given) R^P are isolated residuals;
 * the coarse geometry is the element geometry interpolated to order N.
 * isolated == 0: R^N is the full residual of the coarse discretisation with
 * orders min(N_s, P_e) in every element, and R^P the full residual at P.
 * accumulate != 0 keeps the maximum with the values already in the maps
 * (F_max over estimation stages, Sec. 2.4, approach 2). */
void orc_tau(void* h, const double* q, const double* rP, const int* sweep, int ns, int isolated, int accumulate,
             double* tau_new, double* tau_trad) {
  omesh* m = h;
  const ophys* ph = &m->ph;
  long nsz = NV * m->off[m->n_elem];
  double* RP = malloc(sizeof(double) * nsz);
  if (rP) memcpy(RP, rP, sizeof(double) * nsz);
  else if (!isolated) orc_residual(h, q, RP, 0);
  else {
#pragma omp parallel for schedule(guided)
    for (int e = 0; e < m->n_elem; ++e) isolated_residual(ph, &m->geo[e], q + NV * m->off[e], RP + NV * m->off[e]);
  }
  if (isolated) {
#pragma omp parallel for schedule(guided)
    for (int e = 0; e < m->n_elem; ++e) {
      const int* P = m->ord + 3 * e;
      const double* qP = q + NV * m->off[e];
      const double* rPe = RP + NV * m->off[e];
      for (int s = 0; s < ns; ++s) {
        const int* N = sweep + 3 * s;
        long o = (long)e * ns + s;
        if (N[0] > P[0] || N[1] > P[1] || N[2] > P[2]) { tau_new[o] = -1.0; tau_trad[o] = -1.0; continue; }
        egeo gN;
        elem_geometry(m, e, N, &gN);
        int nN = gN.n;
        double* qN = malloc(sizeof(double) * NV * nN);
        double* RN = malloc(sizeof(double) * NV * nN);
        double* IR = malloc(sizeof(double) * NV * nN);
        interp_elem(P, N, NV, qP, qN);
        interp_elem(P, N, NV, rPe, IR);
        isolated_residual(ph, &gN, qN, RN);
        for (int i = 0; i < NV * nN; ++i) IR[i] -= RN[i];
        double a, b;
        tau_norms(&gN, IR, &a, &b);
        store(tau_new + o, accumulate, a);
        store(tau_trad + o, accumulate, b);
        free(qN); free(RN); free(IR);
        egeo_free(&gN);
      }
    }
  } else {
    int* cord = malloc(sizeof(int) * 3 * m->n_elem);
    for (int s = 0; s < ns; ++s) {
      const int* N = sweep + 3 * s;
      for (int e = 0; e < m->n_elem; ++e)
        for (int d = 0; d < 3; ++d) cord[3 * e + d] = N[d] < m->ord[3 * e + d] ? N[d] : m->ord[3 * e + d];
      omesh* c = orc_mesh_new(m->n_elem, m->G, m->geom, m->nbr, cord, ph->eqs, ph->gamma, ph->mu, ph->Pr, ph->Rgas,
                              ph->qinf);
      long ncs = NV * c->off[c->n_elem];
      double* qc = malloc(sizeof(double) * ncs);
      double* Rc = malloc(sizeof(double) * ncs);
      for (int e = 0; e < m->n_elem; ++e) interp_elem(m->ord + 3 * e, cord + 3 * e, NV, q + NV * m->off[e], qc + NV * c->off[e]);
      orc_residual(c, qc, Rc, 0);
      for (int e = 0; e < m->n_elem; ++e) {
        const int* P = m->ord + 3 * e;
        long o = (long)e * ns + s;
        if (N[0] > P[0] || N[1] > P[1] || N[2] > P[2]) { tau_new[o] = -1.0; tau_trad[o] = -1.0; continue; }
        int nN = c->geo[e].n;
        double* IR = malloc(sizeof(double) * NV * nN);
        interp_elem(P, N, NV, RP + NV * m->off[e], IR);
        for (int i = 0; i < NV * nN; ++i) IR[i] -= Rc[NV * c->off[e] + i];
        double a, b;
        tau_norms(&c->geo[e], IR, &a, &b);
        store(tau_new + o, accumulate, a);
        store(tau_trad + o, accumulate, b);
        free(IR);
      }
      free(qc); free(Rc);
      orc_mesh_free(c);
    }
    free(cord);
  }
  free(RP);
}

/* Element-local isolated residual of a state given at orders N on element e
 * (geometry interpolated to N), for tests of the sweep's building blocks. */
void orc_isolated_residual_at(void* h, int e, const int* N, const double* qN, double* RN) {
  omesh* m = h;
  egeo g;
  elem_geometry(m, e, N, &g);
  isolated_residual(&m->ph, &g, qN, RN);
  egeo_free(&g);
}

/* ------------------------------------------------------------------------ */
/* 9. Projection of the state to new orders (Sec. 2.4: after adaptation the  */
/*    solution is projected to the new polynomial spaces)                    */
/* ------------------------------------------------------------------------ */

/* Per direction: interpolation when the order rises (exact), L2 projection
 * (orc_proj_mat) when it falls. */
void orc_set_orders(void* h, const int* new_ord, const double* q_old, double* q_new) {
  omesh* m = h;
  long off_new = 0;
  for (int e = 0; e < m->n_elem; ++e) {
    const int* No = m->ord + 3 * e;
    const int* Nn = new_ord + 3 * e;
    double* mats[3];
    for (int d = 0; d < 3; ++d) {
      mats[d] = malloc(sizeof(double) * (Nn[d] + 1) * (No[d] + 1));
      if (Nn[d] >= No[d]) orc_interp_mat(No[d], Nn[d], mats[d]);
      else orc_proj_mat(No[d], Nn[d], mats[d]);
    }
    int no = nnodes(No), nn = nnodes(Nn);
    for (int v = 0; v < NV; ++v) apply_3d(mats, No, Nn, q_old + NV * m->off[e] + v * no, q_new + NV * off_new + v * nn);
    off_new += nn;
    for (int d = 0; d < 3; ++d) free(mats[d]);
  }
}

/* ------------------------------------------------------------------------ */
/* 10. Static p-adaptation: order selection from the total truncation-error */
/*     map (Sec. 2.4, approach 2) and the degree-jump conditions (Sec. 3.1)  */
/* ------------------------------------------------------------------------ */

/* For every element: among the sweep entries N with 0 <= map[e][s] < tau_max
 * and n_min <= N_i <= n_max, the one with the fewest degrees of freedom
 * NDOF = prod_i (N_i + 1) (Table 1); the first such entry in sweep order on
 * ties.  With no such entry the element gets n_max in every direction (the
 * secure choice when the error is not known to be below tau_max).
 * Then the jump condition is enforced as the least fixed point above the
 * selection: rule 1 (Eq. N23) N_i^e >= max_j floor(2 N_i^j / 3), rule 2
 * (Eq. N_1) N_i^e >= max_j (N_i^j - 1), over the face neighbours j of e
 * (aligned axes: direction i of the neighbour is direction i of e), rule 0:
 * none.  Orders are raised by Jacobi sweeps until nothing changes. */
void orc_select_orders(int n_elem, int n_sweep, const int* sweep, const double* map, double tau_max, int n_min,
                       int n_max, int jump_rule, const int* nbr, const int* prev, int max_decrease, int* out) {
  for (int e = 0; e < n_elem; ++e) {
    long best = -1;
    int bs = -1;
    for (int s = 0; s < n_sweep; ++s) {
      const double v = map[(long)e * n_sweep + s];
      const int* N = sweep + 3 * s;
      int ok = v >= 0.0 && v < tau_max;
      for (int d = 0; d < 3; ++d) ok = ok && N[d] >= n_min && N[d] <= n_max;
      if (!ok) continue;
      long nd = (long)(N[0] + 1) * (N[1] + 1) * (N[2] + 1);
      if (best < 0 || nd < best) { best = nd; bs = s; }
    }
    for (int d = 0; d < 3; ++d) out[3 * e + d] = bs >= 0 ? sweep[3 * bs + d] : n_max;
    /* dynamic adaptation, Sec. 3.2: an order falls by at most max_decrease
       per adaptation stage */
    if (prev && max_decrease >= 0)
      for (int d = 0; d < 3; ++d) {
        int lo = prev[3 * e + d] - max_decrease;
        if (lo > n_max) lo = n_max;
        if (out[3 * e + d] < lo) out[3 * e + d] = lo;
      }
  }
  if (jump_rule == 0) return;
  int* tmp = malloc(sizeof(int) * 3 * n_elem);
  for (int changed = 1; changed;) {
    changed = 0;
    memcpy(tmp, out, sizeof(int) * 3 * n_elem);
    for (int e = 0; e < n_elem; ++e)
      for (int d = 0; d < 3; ++d) {
        int need = tmp[3 * e + d];
        for (int f = 0; f < 6; ++f) {
          int j = nbr[6 * e + f];
          if (j < 0) continue;
          int nj = tmp[3 * j + d];
          int lim = jump_rule == 1 ? (2 * nj) / 3 : nj - 1;
          if (lim > need) need = lim;
        }
        if (need > out[3 * e + d]) { out[3 * e + d] = need; changed = 1; }
      }
  }
  free(tmp);
}

/* ------------------------------------------------------------------------
 * Truncation-error extrapolation to N_i >= P_i (Sec. 2.3 mentions it, Sec. 2.4
 * needs it for approach 2; the method itself is in the authors' earlier
 * anisotropic work).  The reading used here, step by step, for one element
 * with orders P and its map over the sweep list:
 *   1. directional values: d_i(n) = map at the orders P with N_i = n, for
 *      n = 1 .. P_i - 1 (only the entries present in the sweep);
 *   2. a least-squares line through (n, ln d_i(n)) over the last n_fit of
 *      those points (all of them when n_fit <= 0); the direction is
 *      extrapolable when at least two points are positive and the slope is
 *      negative (exponential decay, the asymptotic range).  Then
 *      e_i(n) = exp(a_i + b_i n) for n >= P_i;
 *   3. d_i(P_i - 1) <= tau_floor (resolved below P: exactly zero when
 *      tau_floor = 0, or at the roundoff level of the estimate): e_i(n) = 0;
 *   4. otherwise e_i(n) = +infinity for n >= P_i (Sec. 2.4, the "high
 *      value" assigned when extrapolation is not possible);
 *   5. the value at a target N:
 *        coupled:   map(min(N, P)) + sum over N_i >= P_i of e_i(N_i), with
 *                   map(P) = 0 and -1 when min(N, P) is not in the sweep;
 *        decoupled: sum_i c_i(N_i), c_i(n) = d_i(n) for n < P_i, e_i(n)
 *                   otherwise (-1 when a needed d_i is missing).
 * out: [n_elem][n_target]; accumulate: out = max(out, value).
 * ---------------------------------------------------------------------- */
static int sweep_find(const int* sweep, int n_sweep, int a, int b, int c) {
  for (int s = 0; s < n_sweep; ++s)
    if (sweep[3 * s] == a && sweep[3 * s + 1] == b && sweep[3 * s + 2] == c) return s;
  return -1;
}

void orc_tau_extrapolate(int n_elem, const int* orders, int n_sweep, const int* sweep, const double* map,
                         int n_target, const int* target, int n_fit, double tau_floor, int decoupled, int accumulate,
                         double* out) {
  for (int e = 0; e < n_elem; ++e) {
    const int* P = orders + 3 * e;
    const double* row = map + (long)e * n_sweep;
    double dv[3][NMAX];      /* directional values, -1 = missing */
    int kind[3];             /* 0: exponential fit, 1: zero, 2: infinity */
    double a[3] = {0, 0, 0}, b[3] = {0, 0, 0};
    for (int i = 0; i < 3; ++i) {
      for (int n = 1; n < P[i]; ++n) {
        int Nn[3] = {P[0], P[1], P[2]};
        Nn[i] = n;
        int s = sweep_find(sweep, n_sweep, Nn[0], Nn[1], Nn[2]);
        dv[i][n] = s >= 0 ? row[s] : -1.0;
      }
      kind[i] = 2;
      if (P[i] >= 2 && dv[i][P[i] - 1] >= 0.0 && dv[i][P[i] - 1] <= tau_floor) {
        kind[i] = 1;
        continue;
      }
      int lo = n_fit > 0 ? P[i] - n_fit : 1;
      if (lo < 1) lo = 1;
      double sx = 0, sy = 0, sxx = 0, sxy = 0;
      int m = 0;
      for (int n = lo; n < P[i]; ++n) {
        if (!(dv[i][n] > 0.0)) continue;
        double y = log(dv[i][n]);
        sx += n; sy += y; sxx += (double)n * n; sxy += n * y;
        ++m;
      }
      if (m < 2) continue;
      double xm = sx / m, ym = sy / m;
      double slope = (sxy - m * xm * ym) / (sxx - m * xm * xm);
      if (!(slope < 0.0)) continue;
      b[i] = slope;
      a[i] = ym - slope * xm;
      kind[i] = 0;
    }
    for (int t = 0; t < n_target; ++t) {
      const int* N = target + 3 * t;
      double v;
      if (!decoupled) {
        int Nc[3];
        for (int i = 0; i < 3; ++i) Nc[i] = N[i] < P[i] ? N[i] : P[i];
        if (Nc[0] == P[0] && Nc[1] == P[1] && Nc[2] == P[2]) {
          v = 0.0;
        } else {
          int s = sweep_find(sweep, n_sweep, Nc[0], Nc[1], Nc[2]);
          v = s >= 0 ? row[s] : -1.0;
        }
        if (v >= 0.0)
          for (int i = 0; i < 3; ++i)
            if (N[i] >= P[i]) v += kind[i] == 0 ? exp(a[i] + b[i] * N[i]) : kind[i] == 1 ? 0.0 : INFINITY;
      } else {
        v = 0.0;
        for (int i = 0; i < 3 && v >= 0.0; ++i) {
          double c;
          if (N[i] < P[i]) c = dv[i][N[i]];
          else c = kind[i] == 0 ? exp(a[i] + b[i] * N[i]) : kind[i] == 1 ? 0.0 : INFINITY;
          v = c < 0.0 ? -1.0 : v + c;
        }
      }
      double* o = out + (long)e * n_target + t;
      *o = accumulate ? (v > *o ? v : *o) : v;
    }
  }
}

/* ------------------------------------------------------------------------
 * The discrete adjoint by brute force, the reference for the adjoint
 * (vector-Jacobian product) kernels: every column of the Jacobian of the
 * residual, or of one RK3 step with dt held fixed, by fourth-order central
 * differences of this file's own functions,
 *   J e_k = (-F(q + 2h e_k) + 8 F(q + h e_k) - 8 F(q - h e_k) + F(q - 2h e_k)) / (12 h),
 * then out_k = v . J e_k.  Column k steps by h = eps * s, s the largest |q|
 * of the column's variable over the mesh (a zero component still gets a
 * sensible step).  The error is O(h^4) plus rounding of order 1e-16 / eps.
 * ---------------------------------------------------------------------- */
static void var_of_dof(const omesh* m, int* var, double s[NV], const double* q) {
  for (int v = 0; v < NV; ++v) s[v] = 0.0;
  for (int e = 0; e < m->n_elem; ++e) {
    const long n = m->off[e + 1] - m->off[e];
    for (int v = 0; v < NV; ++v)
      for (long p = 0; p < n; ++p) {
        const long k = NV * m->off[e] + v * n + p;
        var[k] = v;
        if (fabs(q[k]) > s[v]) s[v] = fabs(q[k]);
      }
  }
  for (int v = 0; v < NV; ++v) if (s[v] == 0.0) s[v] = 1.0;
}

/* which: 0 residual, 1 isolated residual, 2 one RK3 step of size dt */
static void fd_apply(void* h, int which, double dt, const double* x, double* y, double* G, long ns) {
  if (which == 2) {
    memcpy(y, x, sizeof(double) * ns);
    memset(G, 0, sizeof(double) * ns);
    orc_rk_step(h, y, G, dt);
  } else {
    orc_residual(h, x, y, which);
  }
}

static void fd_vjp(void* h, int which, double dt, const double* q, const double* v, double eps, double* out) {
  omesh* m = h;
  const long ns = NV * m->off[m->n_elem];
  int* var = malloc(sizeof(int) * ns);
  double s[NV];
  var_of_dof(m, var, s, q);
  #pragma omp parallel
  {
    double* x = malloc(sizeof(double) * ns);
    double* y = malloc(sizeof(double) * ns);
    double* G = malloc(sizeof(double) * ns);
    double* col = malloc(sizeof(double) * ns);
    memcpy(x, q, sizeof(double) * ns);
    #pragma omp for schedule(dynamic, 4)
    for (long k = 0; k < ns; ++k) {
      const double hk = eps * s[var[k]];
      const double c[4] = {-1.0, 8.0, -8.0, 1.0}, d[4] = {2.0, 1.0, -1.0, -2.0};
      for (long i = 0; i < ns; ++i) col[i] = 0.0;
      for (int t = 0; t < 4; ++t) {
        x[k] = q[k] + d[t] * hk;
        fd_apply(h, which, dt, x, y, G, ns);
        for (long i = 0; i < ns; ++i) col[i] += c[t] * y[i];
      }
      x[k] = q[k];
      double a = 0.0;
      for (long i = 0; i < ns; ++i) a += v[i] * col[i];
      out[k] = a / (12.0 * hk);
    }
    free(x); free(y); free(G); free(col);
  }
  free(var);
}

void orc_residual_vjp_fd(void* h, const double* q, const double* v, double eps, int isolated, double* out) {
  fd_vjp(h, isolated ? 1 : 0, 0.0, q, v, eps, out);
}

void orc_rk_step_vjp_fd(void* h, const double* q, double dt, const double* lam, double eps, double* out) {
  fd_vjp(h, 2, dt, q, lam, eps, out);
}

/* ------------------------------------------------------------------------
 * Force of the fluid on the boundary faces with tag `tag` (the wall of the
 * cylinder case, Sec. 3.3: drag and lift):
 *   F = sum over those faces and their GL nodes of w_a w_b |J a^dir| (p n - tau n),
 * n the unit outward normal of the fluid element (pointing into the body),
 * p the pressure and tau the viscous stress of the node's state and BR1
 * gradient (Navier-Stokes; zero for Euler).  The face's own GL rule.
 * ---------------------------------------------------------------------- */
void orc_wall_force(void* h, const double* q, int tag, double* F) {
  omesh* m = h;
  const ophys* ph = &m->ph;
  double* g = NULL;
  if (ph->eqs == 1) {
    g = malloc(sizeof(double) * 3 * NV * m->off[m->n_elem]);
    orc_gradient(h, q, g, 0);
  }
  F[0] = F[1] = F[2] = 0.0;
  for (int e = 0; e < m->n_elem; ++e)
    for (int f = 0; f < 6; ++f) {
      if (m->nbr[6 * e + f] != tag) continue;
      const int* N = m->ord + 3 * e;
      const egeo* geo = &m->geo[e];
      const int n = geo->n, dir = f / 2, side = f % 2;
      int t0, t1;
      tangential(dir, &t0, &t1);
      double xa[NMAX], wa[NMAX], xb[NMAX], wb[NMAX];
      orc_gl(N[t0], xa, wa);
      orc_gl(N[t1], xb, wb);
      for (int b = 0; b <= N[t1]; ++b)
        for (int a = 0; a <= N[t0]; ++a) {
          const int p = face_vol_index(N, f, a, b);
          double ja[3], nv[3], qn[NV];
          for (int c = 0; c < 3; ++c) ja[c] = geo->Ja[dir][c][p];
          const double area = sqrt(ja[0] * ja[0] + ja[1] * ja[1] + ja[2] * ja[2]);
          for (int c = 0; c < 3; ++c) nv[c] = (side ? 1.0 : -1.0) * ja[c] / area;
          for (int v = 0; v < NV; ++v) qn[v] = q[NV * m->off[e] + v * n + p];
          const double pr = (ph->gamma - 1.0) * (qn[4] - 0.5 * (qn[1] * qn[1] + qn[2] * qn[2] + qn[3] * qn[3]) / qn[0]);
          double tn[3] = {0.0, 0.0, 0.0};
          if (g) {
            double gq[3 * NV], fv[NV];
            for (int v = 0; v < NV; ++v)
              for (int c = 0; c < 3; ++c) gq[v * 3 + c] = g[3 * NV * m->off[e] + (c * NV + v) * n + p];
            for (int d = 0; d < 3; ++d) {
              visc_flux(ph, qn, gq, d, fv);   /* fv[1 + i] = tau_{i d} */
              for (int i = 0; i < 3; ++i) tn[i] += fv[1 + i] * nv[d];
            }
          }
          const double wgt = wa[a] * wb[b] * area;
          for (int i = 0; i < 3; ++i) F[i] += wgt * (pr * nv[i] - tn[i]);
        }
    }
  free(g);
}
