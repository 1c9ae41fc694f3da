// Host construction of the 1D operators (run once per context).  The solution
// and volume quadrature share one node set, GL or LGL; below, xg/wg are those
// nodes and weights whichever set it is.
//
// GL and Lobatto rules by Newton iteration on the Legendre recurrence;
// Lagrange interpolation and differentiation in barycentric form (Berrut &
// Trefethen's formulas); SBP skew operator S1 = W D - D^T W (Sec.
// "Computational Space", SBP property); ESFR K1 = c (D^p)^T W D^p = 2c g g^T,
// g_j the p-th derivative of the j-th Lagrange polynomial (Eq. Km in 1D with
// J = 1); FR projection Pi~1 = (W + K1)^{-1} W (Eq. Fr projection with
// chi = I) written in Sherman-Morrison form, and its inverse I + W^{-1} K1.
#include <cmath>
#include <cstring>
#include <utility>

#include "nsfr_internal.h"

static void legendre(int N, double x, double* P, double* dP) {
  double p0 = 1.0, p1 = x;
  if (N == 0) {
    *P = 1.0;
    *dP = 0.0;
    return;
  }
  for (int k = 2; k <= N; ++k) {
    double p2 = ((2.0 * k - 1.0) * x * p1 - (k - 1.0) * p0) / k;
    p0 = p1;
    p1 = p2;
  }
  *P = p1;
  *dP = (std::fabs(x * x - 1.0) > 0.0) ? N * (x * p1 - p0) / (x * x - 1.0) : 0.0;
}

void nsfr_gauss_legendre(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  for (int i = 0; i < n; ++i) {
    double xi = -std::cos(pi * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, xi, &P, &dP);
      double dx = P / dP;
      xi -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    double P, dP;
    legendre(n, xi, &P, &dP);
    x[i] = xi;
    w[i] = 2.0 / ((1.0 - xi * xi) * dP * dP);
  }
}

void nsfr_gauss_lobatto(int n, double* x, double* w) {
  const double pi = 3.14159265358979323846;
  const int N = n - 1;
  x[0] = -1.0;
  x[N] = 1.0;
  for (int i = 1; i < N; ++i) {
    double xi = -std::cos(pi * i / N);
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(N, xi, &P, &dP);
      double d2P = (2.0 * xi * dP - N * (N + 1.0) * P) / (1.0 - xi * xi);
      double dx = dP / d2P;
      xi -= dx;
      if (std::fabs(dx) < 1e-16) break;
    }
    x[i] = xi;
  }
  for (int i = 0; i < n; ++i) {
    double P, dP;
    legendre(N, x[i], &P, &dP);
    w[i] = 2.0 / (N * (N + 1.0) * P * P);
  }
}

// barycentric weights lambda_j = 1 / prod_{k != j} (x_j - x_k)
static void bary_weights(int n, const double* x, double* lam) {
  for (int j = 0; j < n; ++j) {
    double prod = 1.0;
    for (int k = 0; k < n; ++k)
      if (k != j) prod *= (x[j] - x[k]);
    lam[j] = 1.0 / prod;
  }
}

// L[r][j] = l_j(y_r), r < m: barycentric interpolation matrix (m x n)
static void interp_matrix(int n, const double* x, int m, const double* y, double* L) {
  double lam[NSFR_MAXN];
  bary_weights(n, x, lam);
  for (int r = 0; r < m; ++r) {
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (y[r] == x[j]) hit = j;
    if (hit >= 0) {
      for (int j = 0; j < n; ++j) L[r * n + j] = (j == hit) ? 1.0 : 0.0;
      continue;
    }
    double den = 0.0;
    for (int j = 0; j < n; ++j) den += lam[j] / (y[r] - x[j]);
    for (int j = 0; j < n; ++j) L[r * n + j] = (lam[j] / (y[r] - x[j])) / den;
  }
}

// D[i][j] = l_j'(x_i) on the nodes themselves (barycentric, negative-sum diagonal)
static void diff_matrix(int n, const double* x, double* D) {
  double lam[NSFR_MAXN];
  bary_weights(n, x, lam);
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

void nsfr_build_ops(int p, int p_geo, double c, double gamma, int nodes, OpsGL* gl, OpsGeo* geo) {
  const int n = p + 1;
  const int q = p_geo + 1;
  std::memset(gl, 0, sizeof(*gl));
  std::memset(geo, 0, sizeof(*geo));
  double xg[NSFR_MAXN], wg[NSFR_MAXN], xl[NSFR_MAXN], wl[NSFR_MAXN], xe[NSFR_MAXN];
  nsfr_gauss_lobatto(n, xl, wl);
  // solution = volume quadrature nodes: GL, or LGL (then the face nodes are
  // boundary volume nodes and the extrapolations t_-, t_+ are unit vectors)
  if (nodes == NSFR_NODES_LGL) {
    for (int j = 0; j < n; ++j) {
      xg[j] = xl[j];
      wg[j] = wl[j];
    }
  } else {
    nsfr_gauss_legendre(n, xg, wg);
  }
  for (int k = 0; k < q; ++k) xe[k] = (q == 1) ? 0.0 : -1.0 + 2.0 * k / (q - 1);

  gl->n = n;
  gl->gamma = gamma;
  gl->lgl = (nodes == NSFR_NODES_LGL);
  gl->has_K = (c != 0.0);
  double D[NSFR_MAXN * NSFR_MAXN];
  diff_matrix(n, xg, D);
  double ends[2] = {-1.0, 1.0};
  double T[2 * NSFR_MAXN];
  interp_matrix(n, xg, 2, ends, T);
  for (int j = 0; j < n; ++j) {
    gl->w[j] = wg[j];
    gl->tm[j] = T[j];
    gl->tp[j] = T[n + j];
  }
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) gl->S1[a * n + b] = wg[a] * D[a * n + b] - D[b * n + a] * wg[b];
  // g_j = p! lambda_j (p-th derivative of l_j)
  double lam[NSFR_MAXN], g[NSFR_MAXN];
  bary_weights(n, xg, lam);
  double fact = 1.0;
  for (int k = 2; k <= p; ++k) fact *= k;
  for (int j = 0; j < n; ++j) g[j] = fact * lam[j];
  // K1 = 2 c g g^T ; (W + K1)^{-1} W = I - 2c W^{-1} g g^T / (1 + 2c g^T W^{-1} g)
  double gWg = 0.0;
  for (int j = 0; j < n; ++j) gWg += g[j] * g[j] / wg[j];
  const double denom = 1.0 + 2.0 * c * gWg;
  for (int a = 0; a < n; ++a)
    for (int b = 0; b < n; ++b) {
      double id = (a == b) ? 1.0 : 0.0;
      gl->Pi1[a * n + b] = id - 2.0 * c * (g[a] / wg[a]) * g[b] / denom;
      gl->Pinv1[a * n + b] = id + 2.0 * c * (g[a] / wg[a]) * g[b];
    }
  // rank-one form of the same projection: Pi~1 = I - hv g^T
  for (int a = 0; a < n; ++a) {
    gl->gv[a] = g[a];
    gl->hv[a] = 2.0 * c * (g[a] / wg[a]) / denom;
    gl->gvf[a] = (float)gl->gv[a];
    gl->hvf[a] = (float)gl->hv[a];
  }
  // series of the logarithmic mean in u = f^2, f = (a-b)/(a+b):
  //   atanh(f)/f = 1 + u/3 + u^2/5 + u^3/7 + ...,  f/atanh(f) = 1 - u/3 - 4u^2/45 - 44u^3/945 - ...
  const double F[4] = {1.0, 1.0 / 3.0, 1.0 / 5.0, 1.0 / 7.0};
  const double G[4] = {1.0, -1.0 / 3.0, -4.0 / 45.0, -44.0 / 945.0};
  for (int k = 0; k < 4; ++k) {
    gl->gh[k] = 0.5 * G[k];
    gl->f4g[k] = 2.0 / (gamma - 1.0) * F[k];
    gl->fr2[k] = 2.0 * F[k];
  }
  gl->inv_gm1 = 1.0 / (gamma - 1.0);
  for (int k = 0; k < 3; ++k) {
    gl->lmg[k] = (float)G[k + 1];
    gl->lma[k] = (float)(2.0 * F[k + 1]);
    gl->lmb[k] = (float)(2.0 / (gamma - 1.0) * F[k + 1]);
  }
  {
    auto split = [](double x, float* hl) {
      hl[0] = (float)x;
      hl[1] = (float)(x - (double)hl[0]);
    };
    split(G[1], gl->lmg_ff);
    split(G[2], gl->lmg_ff + 2);
    gl->lmg_ff[4] = (float)G[3];
    split(gl->f4g[1], gl->lmb_ff);
    split(gl->f4g[2], gl->lmb_ff + 2);
    gl->lmb_ff[4] = (float)gl->f4g[3];
    split(gl->fr2[1], gl->lma_ff);
    split(gl->fr2[2], gl->lma_ff + 2);
    gl->lma_ff[4] = (float)gl->fr2[3];
    gl->cab = gl->fr2[0] + gl->f4g[0];
    split(G[1], gl->lmgd_ff);
    split(2.0 * G[2], gl->lmgd_ff + 2);
    gl->lmgd_ff[4] = (float)(3.0 * G[3]);
  }
  {
    const double cab = 2.0 + 2.0 / (gamma - 1.0);
    gl->cab_hi = (float)cab;
    gl->cab_lo = (float)(cab - (double)gl->cab_hi);
  }
  for (int k = 0; k < n * n; ++k) {
    gl->S1f[k] = (float)gl->S1[k];
  }
  for (int j = 0; j < n; ++j) {
    gl->tmf[j] = (float)gl->tm[j];
    gl->tpf[j] = (float)gl->tp[j];
    gl->tmlo[j] = (float)(gl->tm[j] - (double)gl->tmf[j]);
    gl->tplo[j] = (float)(gl->tp[j] - (double)gl->tpf[j]);
  }
  for (int k = 0; k < n * n; ++k) gl->S1lo[k] = (float)(gl->S1[k] - (double)gl->S1f[k]);

  geo->n = n;
  geo->q = q;
  geo->nq = n;
  interp_matrix(q, xe, n, xl, geo->E);
  interp_matrix(q, xe, n, xg, geo->Eg);
  diff_matrix(n, xl, geo->Dl);
  interp_matrix(n, xl, n, xg, geo->I);
  for (int j = 0; j < n; ++j) geo->w[j] = wg[j];
  gl->uncol = 0;
  gl->ns = n;
}

// X = A^{-1} B for an m x m matrix A and m x k B (Gaussian elimination with
// partial pivoting; m <= NSFR_MAXN); A and B are overwritten
static void solve_small(int m, int k, double* A, double* B) {
  for (int c = 0; c < m; ++c) {
    int piv = c;
    for (int r = c + 1; r < m; ++r)
      if (std::fabs(A[r * m + c]) > std::fabs(A[piv * m + c])) piv = r;
    if (piv != c) {
      for (int j = 0; j < m; ++j) std::swap(A[c * m + j], A[piv * m + j]);
      for (int j = 0; j < k; ++j) std::swap(B[c * k + j], B[piv * k + j]);
    }
    for (int r = c + 1; r < m; ++r) {
      const double f = A[r * m + c] / A[c * m + c];
      for (int j = c; j < m; ++j) A[r * m + j] -= f * A[c * m + j];
      for (int j = 0; j < k; ++j) B[r * k + j] -= f * B[c * k + j];
    }
  }
  for (int c = m - 1; c >= 0; --c)
    for (int j = 0; j < k; ++j) {
      double v = B[c * k + j];
      for (int i = c + 1; i < m; ++i) v -= A[c * m + i] * B[i * k + j];
      B[c * k + j] = v / A[c * m + c];
    }
}

// Uncollocated operators (the scheme of the paper's runs: solution on the p+1
// Lobatto nodes, volume and face quadrature on nq >= p+1 Gauss-Legendre
// points).  The line kernels see the GL points: their derivative D_q = chi D
// Pi, S_q = W D_q - D_q^T W and extrapolations E_-+ = l(-+1)^T Pi satisfy
// W D_q + D_q^T W = E+^T E+ - E-^T E- (the quadrature integrates degree 2p).
void nsfr_build_ops_uncol(int p, int p_geo, int nq, double c, double gamma, OpsGL* gl, OpsGeo* geo) {
  const int ns = p + 1, q = p_geo + 1;
  // the collocated GL operators of nq points give the series constants and layout
  nsfr_build_ops(nq - 1, p_geo < nq - 1 ? p_geo : nq - 1, 0.0, gamma, NSFR_NODES_GL, gl, geo);
  double xl[NSFR_MAXN], wl[NSFR_MAXN], xq[NSFR_MAXN], wq[NSFR_MAXN], xe[NSFR_MAXN];
  nsfr_gauss_lobatto(ns, xl, wl);
  nsfr_gauss_legendre(nq, xq, wq);
  for (int k = 0; k < q; ++k) xe[k] = (q == 1) ? 0.0 : -1.0 + 2.0 * k / (q - 1);
  double chi[NSFR_MAXN * NSFR_MAXN], D[NSFR_MAXN * NSFR_MAXN];
  interp_matrix(ns, xl, nq, xq, chi);  // nq x ns
  diff_matrix(ns, xl, D);
  double ends[2] = {-1.0, 1.0}, L[2 * NSFR_MAXN];
  interp_matrix(ns, xl, 2, ends, L);
  // M1 = chi^T W chi, Pi = M1^{-1} chi^T W
  double M1[NSFR_MAXN * NSFR_MAXN], Pi[NSFR_MAXN * NSFR_MAXN], tmp[NSFR_MAXN * NSFR_MAXN];
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b) {
      double v = 0.0;
      for (int r = 0; r < nq; ++r) v += chi[r * ns + a] * wq[r] * chi[r * ns + b];
      M1[a * ns + b] = v;
    }
  for (int a = 0; a < ns; ++a)
    for (int r = 0; r < nq; ++r) Pi[a * nq + r] = chi[r * ns + a] * wq[r];
  std::memcpy(tmp, M1, sizeof(tmp));
  solve_small(ns, nq, tmp, Pi);
  // D_q = chi D Pi (nq x nq)
  double DPi[NSFR_MAXN * NSFR_MAXN], Dq[NSFR_MAXN * NSFR_MAXN];
  for (int a = 0; a < ns; ++a)
    for (int r = 0; r < nq; ++r) {
      double v = 0.0;
      for (int b = 0; b < ns; ++b) v += D[a * ns + b] * Pi[b * nq + r];
      DPi[a * nq + r] = v;
    }
  for (int r = 0; r < nq; ++r)
    for (int t = 0; t < nq; ++t) {
      double v = 0.0;
      for (int a = 0; a < ns; ++a) v += chi[r * ns + a] * DPi[a * nq + t];
      Dq[r * nq + t] = v;
    }
  gl->uncol = 1;
  gl->ns = ns;
  gl->has_K = (c != 0.0);
  for (int r = 0; r < nq; ++r)
    for (int t = 0; t < nq; ++t) gl->S1[r * nq + t] = wq[r] * Dq[r * nq + t] - Dq[t * nq + r] * wq[t];
  for (int r = 0; r < nq; ++r) {
    double em = 0.0, ep = 0.0;
    for (int a = 0; a < ns; ++a) {
      em += L[a] * Pi[a * nq + r];
      ep += L[ns + a] * Pi[a * nq + r];
    }
    gl->tm[r] = em;
    gl->tp[r] = ep;
    gl->w[r] = wq[r];
  }
  std::memcpy(gl->chi, chi, sizeof(gl->chi));
  std::memcpy(gl->Pi, Pi, sizeof(gl->Pi));
  for (int a = 0; a < ns; ++a) {
    gl->ls_m[a] = L[a];
    gl->ls_p[a] = L[ns + a];
  }
  // Pi~1 = (M1 + K1)^{-1} chi^T W, K1 = c (D^p)^T M1 D^p = 2c g g^T (rows of D^p are g^T)
  double lam[NSFR_MAXN], g[NSFR_MAXN];
  bary_weights(ns, xl, lam);
  double fact = 1.0;
  for (int k = 2; k <= p; ++k) fact *= k;
  for (int j = 0; j < ns; ++j) g[j] = fact * lam[j];
  double MK[NSFR_MAXN * NSFR_MAXN], Pt[NSFR_MAXN * NSFR_MAXN];
  for (int a = 0; a < ns; ++a)
    for (int b = 0; b < ns; ++b) MK[a * ns + b] = M1[a * ns + b] + 2.0 * c * g[a] * g[b];
  for (int a = 0; a < ns; ++a)
    for (int r = 0; r < nq; ++r) Pt[a * nq + r] = chi[r * ns + a] * wq[r];
  solve_small(ns, nq, MK, Pt);
  std::memcpy(gl->Pt, Pt, sizeof(gl->Pt));
  // A = (chi Pi~1)^T, nq x nq
  for (int r = 0; r < nq; ++r)
    for (int t = 0; t < nq; ++t) {
      double v = 0.0;
      for (int a = 0; a < ns; ++a) v += chi[t * ns + a] * Pt[a * nq + r];
      gl->A[r * nq + t] = v;
    }
  // FP32 (and float-float) copies of what this function replaced, for the FP32-bulk kernel
  for (int k = 0; k < nq * nq; ++k) {
    gl->S1f[k] = (float)gl->S1[k];
    gl->S1lo[k] = (float)(gl->S1[k] - (double)gl->S1f[k]);
  }
  for (int j = 0; j < nq; ++j) {
    gl->tmf[j] = (float)gl->tm[j];
    gl->tpf[j] = (float)gl->tp[j];
    gl->tmlo[j] = (float)(gl->tm[j] - (double)gl->tmf[j]);
    gl->tplo[j] = (float)(gl->tp[j] - (double)gl->tpf[j]);
  }
  for (int k = 0; k < NSFR_MAXN * NSFR_MAXN; ++k) {
    gl->chif[k] = (float)gl->chi[k];
    gl->Af[k] = (float)gl->A[k];
    gl->Ptf[k] = (float)gl->Pt[k];
  }
  // metric construction: degree-p Lobatto layer, evaluated at the GL points;
  // node coordinates at the Lobatto solution nodes
  geo->n = ns;
  geo->q = q;
  geo->nq = nq;
  interp_matrix(q, xe, ns, xl, geo->E);
  interp_matrix(q, xe, ns, xl, geo->Eg);
  diff_matrix(ns, xl, geo->Dl);
  interp_matrix(ns, xl, nq, xq, geo->I);
  for (int r = 0; r < nq; ++r) geo->w[r] = wq[r];
}
