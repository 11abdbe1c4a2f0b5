// Dense FP64 linear algebra of the factor step and the check that the
// general per-node recursion of the dual gradient collapses to the single
// shared operator that the kernels apply.
//
// The dual gradient x*(w) (paper §4.4, eq. dual-gradient) solves an
// equality-constrained QP on the scenario tree by a Riccati-type recursion
// from the leaves up.  With L an orthonormal basis of ker E it reads, per
// node nu with children c:
//   Q_nu   = 2 p_nu W_u + sum_c P_c
//   Phi_nu = L (L' Q_nu L)^-1 L'
//   P_nu   = 2 p_nu W_u - (2 p_nu W_u) Phi_nu (2 p_nu W_u)
// The kernels use instead one operator for every node,
//   F = W^-1 - W^-1 E' S^-1 E W^-1,  S = E W^-1 E'  (W = W_u, diagonal or dense),
// with Phi_nu = F / (2 p_nu).  That is exact by induction from the leaves:
// F = L (L' W L)^-1 L', so a leaf (Q = 2 p W) has 2 p Phi = F; and when
// every child has Phi_c = F / (2 p_c), then P_c = 2 p_c (W - W F W), which
// L' (.) L annihilates because L' W F W L = L' W L, so L' Q_nu L =
// 2 p_nu L' W L again.  collapse_deviation evaluates this step in floating
// point with the F the factor step computed and the tree's actual
// probabilities, at a leaf and at interior nodes.
#include <algorithm>
#include <cmath>

#include "rn_internal.h"

namespace rn {

bool cholesky(std::vector<double> &A, int m) {
  double scale = 0.0;
  for (int i = 0; i < m; ++i) scale = std::max(scale, std::fabs(A[(size_t)i * m + i]));
  for (int j = 0; j < m; ++j) {
    double d = A[(size_t)j * m + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * m + k] * A[(size_t)j * m + k];
    if (!(d > 1e-13 * scale)) return false;
    d = std::sqrt(d);
    A[(size_t)j * m + j] = d;
    for (int i = j + 1; i < m; ++i) {
      double v = A[(size_t)i * m + j];
      for (int k = 0; k < j; ++k) v -= A[(size_t)i * m + k] * A[(size_t)j * m + k];
      A[(size_t)i * m + j] = v / d;
    }
  }
  return true;
}

std::vector<double> chol_inverse(const std::vector<double> &R, int m) {
  std::vector<double> inv((size_t)m * m, 0.0), col(m);
  for (int c = 0; c < m; ++c) {
    for (int i = 0; i < m; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= R[(size_t)i * m + k] * col[k];
      col[i] = v / R[(size_t)i * m + i];
    }
    for (int i = m - 1; i >= 0; --i) {
      double v = col[i];
      for (int k = i + 1; k < m; ++k) v -= R[(size_t)k * m + i] * col[k];
      col[i] = v / R[(size_t)i * m + i];
    }
    for (int i = 0; i < m; ++i) inv[(size_t)i * m + c] = col[i];
  }
  return inv;
}

namespace {

// Orthonormal basis of ker E (nu x (nu - ne), row-major) from Householder
// reflections of E' (nu x ne): the last nu - ne columns of Q in E' = Q R.
// Empty if E' has a column that the reflections reduce to zero.
std::vector<double> kernel_basis(const double *E, int ne, int nu) {
  std::vector<double> A((size_t)nu * ne), Q((size_t)nu * nu, 0.0), v(nu);
  for (int r = 0; r < ne; ++r)
    for (int j = 0; j < nu; ++j) A[(size_t)j * ne + r] = E[(size_t)r * nu + j];
  for (int i = 0; i < nu; ++i) Q[(size_t)i * nu + i] = 1.0;
  double scale = 0.0;
  for (double a : A) scale = std::max(scale, std::fabs(a));
  for (int k = 0; k < ne; ++k) {
    double nrm = 0.0;
    for (int i = k; i < nu; ++i) nrm += A[(size_t)i * ne + k] * A[(size_t)i * ne + k];
    nrm = std::sqrt(nrm);
    if (!(nrm > 1e-12 * scale)) return {};
    const double a0 = A[(size_t)k * ne + k];
    const double alpha = a0 > 0 ? -nrm : nrm;
    std::fill(v.begin(), v.end(), 0.0);
    for (int i = k; i < nu; ++i) v[i] = A[(size_t)i * ne + k];
    v[k] -= alpha;
    double vv = 0.0;
    for (int i = k; i < nu; ++i) vv += v[i] * v[i];
    if (vv == 0.0) continue;
    // A <- H A on columns k.., Q <- Q H, with H = I - 2 v v' / (v' v)
    for (int c = k; c < ne; ++c) {
      double s = 0.0;
      for (int i = k; i < nu; ++i) s += v[i] * A[(size_t)i * ne + c];
      s *= 2.0 / vv;
      for (int i = k; i < nu; ++i) A[(size_t)i * ne + c] -= s * v[i];
    }
    for (int r = 0; r < nu; ++r) {
      double s = 0.0;
      for (int i = k; i < nu; ++i) s += Q[(size_t)r * nu + i] * v[i];
      s *= 2.0 / vv;
      for (int i = k; i < nu; ++i) Q[(size_t)r * nu + i] -= s * v[i];
    }
  }
  const int nv = nu - ne;
  std::vector<double> L((size_t)nu * nv);
  for (int r = 0; r < nu; ++r)
    for (int c = 0; c < nv; ++c) L[(size_t)r * nv + c] = Q[(size_t)r * nu + ne + c];
  return L;
}

// C (m x n) = A (m x k) B (k x n), row-major
void matmul(const double *A, const double *B, double *C, int m, int k, int n) {
  std::fill(C, C + (size_t)m * n, 0.0);
  for (int i = 0; i < m; ++i) {
    double *c = C + (size_t)i * n;
    for (int p = 0; p < k; ++p) {
      const double a = A[(size_t)i * k + p];
      if (a == 0.0) continue;
      const double *b = B + (size_t)p * n;
      for (int j = 0; j < n; ++j) c[j] += a * b[j];
    }
  }
}

// C (m x n) = A' B with A (k x m), B (k x n), row-major
void matmul_tn(const double *A, const double *B, double *C, int k, int m, int n) {
  std::fill(C, C + (size_t)m * n, 0.0);
  for (int p = 0; p < k; ++p) {
    const double *a = A + (size_t)p * m, *b = B + (size_t)p * n;
    for (int i = 0; i < m; ++i) {
      const double ai = a[i];
      if (ai == 0.0) continue;
      double *c = C + (size_t)i * n;
      for (int j = 0; j < n; ++j) c[j] += ai * b[j];
    }
  }
}

}  // namespace

double collapse_deviation(const rn_tree *tree, int nu, int ne, const double *E,
                          const double *winv, const double *Sinv) {
  if (nu - ne <= 0) return 0.0;  // u is fixed by E u + Ed d = 0: nothing to factor
  // F (dense, nu x nu) from the same W^-1 and S^-1 the kernels receive
  std::vector<double> EW((size_t)std::max(1, ne) * nu), F((size_t)nu * nu, 0.0);
  for (int r = 0; r < ne; ++r)
    for (int j = 0; j < nu; ++j) EW[(size_t)r * nu + j] = E[(size_t)r * nu + j] * winv[j];
  std::vector<double> T((size_t)std::max(1, ne) * nu, 0.0);  // S^-1 E W^-1
  for (int r = 0; r < ne; ++r)
    for (int s = 0; s < ne; ++s) {
      const double a = Sinv[(size_t)r * ne + s];
      for (int j = 0; j < nu; ++j) T[(size_t)r * nu + j] += a * EW[(size_t)s * nu + j];
    }
  for (int i = 0; i < nu; ++i) {
    F[(size_t)i * nu + i] = winv[i];
    for (int r = 0; r < ne; ++r) {
      const double a = EW[(size_t)r * nu + i];
      if (a == 0.0) continue;
      for (int j = 0; j < nu; ++j) F[(size_t)i * nu + j] -= a * T[(size_t)r * nu + j];
    }
  }
  std::vector<double> W((size_t)nu * nu, 0.0);
  for (int i = 0; i < nu; ++i) W[(size_t)i * nu + i] = 1.0 / winv[i];
  return collapse_deviation_dense(tree, nu, ne, E, W.data(), F.data());
}

double collapse_deviation_dense(const rn_tree *tree, int nu, int ne, const double *E,
                                const double *W, const double *Fp) {
  const int nv = nu - ne, N = tree->N;
  if (nv <= 0) return 0.0;
  const std::vector<double> F(Fp, Fp + (size_t)nu * nu);
  double fmax = 0.0;
  for (double a : F) fmax = std::max(fmax, std::fabs(a));
  std::vector<double> L;
  if (ne > 0) {
    L = kernel_basis(E, ne, nu);
    if (L.empty()) return INFINITY;
  } else {
    L.assign((size_t)nu * nu, 0.0);
    for (int i = 0; i < nu; ++i) L[(size_t)i * nu + i] = 1.0;
  }
  std::vector<double> Lt((size_t)nv * nu);
  for (int i = 0; i < nu; ++i)
    for (int c = 0; c < nv; ++c) Lt[(size_t)c * nu + i] = L[(size_t)i * nv + c];
  // D = W - W F W: a child's P_c / (2 p_c) under the induction hypothesis.
  // L' Q L = 2 p_v L'W L + 2 (sum of the children's p) L'D L.
  std::vector<double> D((size_t)nu * nu), WL((size_t)nu * nv), DL((size_t)nu * nv);
  std::vector<double> WF((size_t)nu * nu), WFW((size_t)nu * nu);
  matmul(W, F.data(), WF.data(), nu, nu, nu);
  matmul(WF.data(), W, WFW.data(), nu, nu, nu);
  for (size_t e = 0; e < D.size(); ++e) D[e] = W[e] - WFW[e];
  matmul(W, L.data(), WL.data(), nu, nu, nv);
  matmul(D.data(), L.data(), DL.data(), nu, nu, nv);
  std::vector<double> LWL((size_t)nv * nv), LDL((size_t)nv * nv);
  matmul_tn(L.data(), WL.data(), LWL.data(), nu, nv, nv);
  matmul_tn(L.data(), DL.data(), LDL.data(), nu, nv, nv);
  // sampled nodes: the first node of stage 1, of the middle stage and of
  // stage N (a leaf, as every leaf is at stage N)
  std::vector<int> sample;
  for (int t : {1, (N + 1) / 2, N}) {
    const int v = tree->stage_ptr[t];
    if (std::find(sample.begin(), sample.end(), v) == sample.end()) sample.push_back(v);
  }
  double worst = 0.0;
  std::vector<double> M((size_t)nv * nv), LM((size_t)nu * nv), Phi((size_t)nu * nu);
  for (int v : sample) {
    int t = 0;
    while (tree->stage_ptr[t + 1] <= v) ++t;
    const double pv = tree->prob[v];
    double pc = 0.0;  // sum of the children's probabilities (0 at a leaf)
    if (t < N)
      for (int c = tree->stage_ptr[t + 1]; c < tree->stage_ptr[t + 2]; ++c)
        if (tree->anc[c] == v) pc += tree->prob[c];
    for (size_t e = 0; e < M.size(); ++e) M[e] = 2.0 * pv * LWL[e] + 2.0 * pc * LDL[e];
    if (!cholesky(M, nv)) return INFINITY;
    const std::vector<double> Mi = chol_inverse(M, nv);
    // 2 p_v Phi_v = 2 p_v L M^-1 L', compared with F
    matmul(L.data(), Mi.data(), LM.data(), nu, nv, nv);
    matmul(LM.data(), Lt.data(), Phi.data(), nu, nv, nu);
    for (size_t e = 0; e < Phi.size(); ++e)
      worst = std::max(worst, std::fabs(2.0 * pv * Phi[e] - F[e]) / fmax);
  }
  return worst;
}

}  // namespace rn
