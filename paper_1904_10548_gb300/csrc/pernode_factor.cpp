// Factor step of the per-node form of the dual gradient (paper §4.4): the
// general Riccati-type recursion with one set of matrices per node, FP64 on
// the host.
//
// The cost-to-go of node nu as a function of its ancestor's (x_a, u_a) is
// linear in x_a (no quadratic state cost) and quadratic in u_a, with the
// Hessian P_nu.  Going from stage N down to stage 1:
//   Q_nu   = 2 p_nu W_u + sum over children c of P_c
//   Phi_nu = L (L' Q_nu L)^-1 L'            (L: orthonormal basis of ker E)
//   K_nu   = Phi_nu (2 p_nu W_u)
//   Mc_nu  = (I - Phi_nu Q_nu) E'           (acts on the coupling's data)
//   P_nu   = 2 p_nu W_u - (2 p_nu W_u) Phi_nu (2 p_nu W_u)
// L' Q L = C C' (Cholesky) gives Phi = Y Y' with Y = L C^-T, and
// P = W2 - (W2 Y)(W2 Y)'.  None of these depends on A: the state matrix
// enters only the vector recursion of every evaluation.
//
// The particular solution of E u + Ed d = 0 is taken in range(E'):
// ud = E' s with s = Sd d, Sd = -(E E')^-1 Ed.  (I - Phi Q) vanishes on
// ker E, so (I - Phi Q) ud = Mc s whatever particular solution is chosen,
// and the per-solve constant of every node is mc = Mc (Sd d), an ne-wide
// product instead of an nu-wide one.
#include <algorithm>
#include <cmath>
#include <thread>
#include <vector>

#include "pernode.h"

namespace rn {
namespace {

// Householder QR of E' (nu x ne): R (ne x ne, upper) and the trailing
// nu - ne columns of Q (an orthonormal basis of ker E, nu x nv row-major).
// false when E does not have full row rank.
bool kernel_basis(const double *E, int ne, int nu, std::vector<double> &L,
                  std::vector<double> &R) {
  const int nv = nu - ne;
  std::vector<double> A((size_t)nu * ne);  // E' row-major
  for (int i = 0; i < nu; ++i)
    for (int k = 0; k < ne; ++k) A[(size_t)i * ne + k] = E[(size_t)k * nu + i];
  std::vector<double> V((size_t)nu * ne, 0.0), beta(ne, 0.0);
  double scale = 0.0;
  for (double a : A) scale = std::max(scale, std::fabs(a));
  for (int k = 0; k < ne; ++k) {
    double nrm = 0.0;
    for (int i = k; i < nu; ++i) nrm += A[(size_t)i * ne + k] * A[(size_t)i * ne + k];
    nrm = std::sqrt(nrm);
    if (!(nrm > 1e-12 * scale)) return false;
    const double a0 = A[(size_t)k * ne + k];
    const double alpha = a0 >= 0.0 ? -nrm : nrm;
    // v = x - alpha e_k, H = I - beta v v'
    double vv = 0.0;
    for (int i = k; i < nu; ++i) {
      const double vi = A[(size_t)i * ne + k] - (i == k ? alpha : 0.0);
      V[(size_t)i * ne + k] = vi;
      vv += vi * vi;
    }
    beta[k] = vv > 0.0 ? 2.0 / vv : 0.0;
    for (int j = k; j < ne; ++j) {
      double dot = 0.0;
      for (int i = k; i < nu; ++i) dot += V[(size_t)i * ne + k] * A[(size_t)i * ne + j];
      dot *= beta[k];
      for (int i = k; i < nu; ++i) A[(size_t)i * ne + j] -= dot * V[(size_t)i * ne + k];
    }
  }
  R.assign((size_t)std::max(1, ne * ne), 0.0);
  double rmax = 0.0;
  for (int k = 0; k < ne; ++k)
    for (int j = k; j < ne; ++j) {
      R[(size_t)k * ne + j] = A[(size_t)k * ne + j];
      rmax = std::max(rmax, std::fabs(A[(size_t)k * ne + j]));
    }
  for (int k = 0; k < ne; ++k)
    if (!(std::fabs(R[(size_t)k * ne + k]) > 1e-12 * rmax)) return false;
  // Q e_j = H_0 H_1 ... H_{ne-1} e_j for the columns j = ne .. nu-1
  L.assign((size_t)nu * std::max(1, nv), 0.0);
  std::vector<double> q(nu);
  for (int c = 0; c < nv; ++c) {
    std::fill(q.begin(), q.end(), 0.0);
    q[ne + c] = 1.0;
    for (int k = ne - 1; k >= 0; --k) {
      double dot = 0.0;
      for (int i = k; i < nu; ++i) dot += V[(size_t)i * ne + k] * q[i];
      dot *= beta[k];
      for (int i = k; i < nu; ++i) q[i] -= dot * V[(size_t)i * ne + k];
    }
    for (int i = 0; i < nu; ++i) L[(size_t)i * nv + c] = q[i];
  }
  return true;
}

// C C' = M (m x m, lower C in place); false unless every pivot is positive
// relative to the diagonal scale
bool chol_lower(double *M, int m) {
  double dmax = 0.0;
  for (int i = 0; i < m; ++i) dmax = std::max(dmax, std::fabs(M[(size_t)i * m + i]));
  for (int j = 0; j < m; ++j) {
    double d = M[(size_t)j * m + j];
    for (int k = 0; k < j; ++k) d -= M[(size_t)j * m + k] * M[(size_t)j * m + k];
    if (!(d > 1e-14 * dmax)) return false;
    const double c = std::sqrt(d);
    M[(size_t)j * m + j] = c;
    const double ic = 1.0 / c;
    for (int i = j + 1; i < m; ++i) {
      double s = M[(size_t)i * m + j];
      const double *ri = M + (size_t)i * m, *rj = M + (size_t)j * m;
      for (int k = 0; k < j; ++k) s -= ri[k] * rj[k];
      M[(size_t)i * m + j] = s * ic;
    }
  }
  return true;
}

struct NodeWork {
  int nu, ne, nv;
  const double *Wu, *L, *Et;  // W_u (nu x nu), L (nu x nv), E' (nu x ne)
  // scratch
  std::vector<double> Q, QL, LQL, Y, W2Y, QE;
  void init() {
    Q.resize((size_t)nu * nu);
    QL.resize((size_t)nu * nv);
    LQL.resize((size_t)nv * nv);
    Y.resize((size_t)nu * nv);
    W2Y.resize((size_t)nu * nv);
    QE.resize((size_t)nu * std::max(1, ne));
  }
  // one node: children's P summed into Q, then Phi, K, Mc and P
  bool run(double p, const double *const *Pc, int nc, double *Phi, double *K, double *Mc,
           double *P) {
    const double w2 = 2.0 * p;
    for (size_t e = 0; e < (size_t)nu * nu; ++e) Q[e] = w2 * Wu[e];
    for (int c = 0; c < nc; ++c)
      for (size_t e = 0; e < (size_t)nu * nu; ++e) Q[e] += Pc[c][e];
    // QL = Q L
    std::fill(QL.begin(), QL.end(), 0.0);
    for (int i = 0; i < nu; ++i) {
      double *qi = &QL[(size_t)i * nv];
      for (int k = 0; k < nu; ++k) {
        const double a = Q[(size_t)i * nu + k];
        if (a == 0.0) continue;
        const double *lk = L + (size_t)k * nv;
        for (int j = 0; j < nv; ++j) qi[j] += a * lk[j];
      }
    }
    // LQL = L' QL (lower triangle, mirrored)
    std::fill(LQL.begin(), LQL.end(), 0.0);
    for (int k = 0; k < nu; ++k) {
      const double *lk = L + (size_t)k * nv, *qk = &QL[(size_t)k * nv];
      for (int i = 0; i < nv; ++i) {
        const double a = lk[i];
        if (a == 0.0) continue;
        double *ri = &LQL[(size_t)i * nv];
        for (int j = 0; j <= i; ++j) ri[j] += a * qk[j];
      }
    }
    for (int i = 0; i < nv; ++i)
      for (int j = i + 1; j < nv; ++j) LQL[(size_t)i * nv + j] = LQL[(size_t)j * nv + i];
    if (!chol_lower(LQL.data(), nv)) return false;
    // Y = L C^-T: each row y of Y solves C y' = l' (forward substitution)
    for (int r = 0; r < nu; ++r) {
      const double *l = L + (size_t)r * nv;
      double *y = &Y[(size_t)r * nv];
      for (int i = 0; i < nv; ++i) {
        double s = l[i];
        const double *ci = &LQL[(size_t)i * nv];
        for (int k = 0; k < i; ++k) s -= ci[k] * y[k];
        y[i] = s / ci[i];
      }
    }
    // Phi = Y Y' (symmetric)
    for (int i = 0; i < nu; ++i) {
      const double *yi = &Y[(size_t)i * nv];
      for (int j = 0; j <= i; ++j) {
        const double *yj = &Y[(size_t)j * nv];
        double s = 0.0;
        for (int k = 0; k < nv; ++k) s += yi[k] * yj[k];
        Phi[(size_t)i * nu + j] = s;
        Phi[(size_t)j * nu + i] = s;
      }
    }
    // K = Phi (2 p W_u)
    for (int i = 0; i < nu; ++i) {
      double *ki = K + (size_t)i * nu;
      std::fill(ki, ki + nu, 0.0);
      for (int k = 0; k < nu; ++k) {
        const double a = Phi[(size_t)i * nu + k] * w2;
        const double *wk = Wu + (size_t)k * nu;
        for (int j = 0; j < nu; ++j) ki[j] += a * wk[j];
      }
    }
    // Mc = E' - Phi (Q E')
    if (ne > 0) {
      std::fill(QE.begin(), QE.end(), 0.0);
      for (int i = 0; i < nu; ++i)
        for (int k = 0; k < nu; ++k) {
          const double a = Q[(size_t)i * nu + k];
          if (a == 0.0) continue;
          for (int j = 0; j < ne; ++j) QE[(size_t)i * ne + j] += a * Et[(size_t)k * ne + j];
        }
      for (int i = 0; i < nu; ++i)
        for (int j = 0; j < ne; ++j) {
          double s = Et[(size_t)i * ne + j];
          for (int k = 0; k < nu; ++k) s -= Phi[(size_t)i * nu + k] * QE[(size_t)k * ne + j];
          Mc[(size_t)i * ne + j] = s;
        }
    }
    // P = W2 - (W2 Y)(W2 Y)'
    if (P) {
      std::fill(W2Y.begin(), W2Y.end(), 0.0);
      for (int i = 0; i < nu; ++i) {
        double *wi = &W2Y[(size_t)i * nv];
        for (int k = 0; k < nu; ++k) {
          const double a = w2 * Wu[(size_t)i * nu + k];
          if (a == 0.0) continue;
          const double *yk = &Y[(size_t)k * nv];
          for (int j = 0; j < nv; ++j) wi[j] += a * yk[j];
        }
      }
      for (int i = 0; i < nu; ++i) {
        const double *ai = &W2Y[(size_t)i * nv];
        for (int j = 0; j <= i; ++j) {
          const double *aj = &W2Y[(size_t)j * nv];
          double s = 0.0;
          for (int k = 0; k < nv; ++k) s += ai[k] * aj[k];
          const double v = w2 * Wu[(size_t)i * nu + j] - s;
          P[(size_t)i * nu + j] = v;
          P[(size_t)j * nu + i] = v;
        }
      }
    }
    return true;
  }
};

}  // namespace

int pn_factor_host(const rn_network *net, const rn_tree *tree, const rn_cost *cost,
                   int threads, PnSink sink, void *ctx, std::vector<double> *Sd_out) {
  const int nu = net->nu, ne = net->ne, nd = net->nd, N = tree->N, n = tree->n_nodes;
  const int nv = nu - ne;
  if (nv < 1) {
    set_error("per-node factor: ne = %d leaves no free inputs (nu = %d)", ne, nu);
    return RN_ERR_RANK;
  }
  std::vector<double> L, R;
  if (ne > 0) {
    if (!kernel_basis(net->E, ne, nu, L, R)) {
      set_error("E does not have full row rank");
      return RN_ERR_RANK;
    }
  } else {
    L.assign((size_t)nu * nu, 0.0);
    for (int i = 0; i < nu; ++i) L[(size_t)i * nu + i] = 1.0;
  }
  // Sd = -(E E')^-1 Ed = -(R' R)^-1 Ed
  if (Sd_out) {
    Sd_out->assign((size_t)std::max(1, ne * nd), 0.0);
    for (int c = 0; c < nd && ne > 0; ++c) {
      std::vector<double> z(ne);
      for (int i = 0; i < ne; ++i) {  // R' z = Ed[:, c]
        double s = net->Ed[(size_t)i * nd + c];
        for (int k = 0; k < i; ++k) s -= R[(size_t)k * ne + i] * z[k];
        z[i] = s / R[(size_t)i * ne + i];
      }
      for (int i = ne - 1; i >= 0; --i) {  // R s = z
        double s = z[i];
        for (int k = i + 1; k < ne; ++k) s -= R[(size_t)i * ne + k] * z[k];
        z[i] = s / R[(size_t)i * ne + i];
      }
      for (int i = 0; i < ne; ++i) (*Sd_out)[(size_t)i * nd + c] = -z[i];
    }
  }
  std::vector<double> Et((size_t)nu * std::max(1, ne), 0.0);
  for (int i = 0; i < nu; ++i)
    for (int k = 0; k < ne; ++k) Et[(size_t)i * ne + k] = net->E[(size_t)k * nu + i];
  // children ranges (children are contiguous and in parent order)
  std::vector<int> cbeg(n, 0), cend(n, 0);
  for (int v = 1; v < n; ++v) {
    const int a = tree->anc[v];
    if (cend[a] == 0) cbeg[a] = v;
    cend[a] = v + 1;
  }
  const size_t mm = (size_t)nu * nu;
  std::vector<double> Pbelow, Phere;  // P of the stage below / this stage
  int below0 = 0;
  threads = std::max(1, threads);
  for (int t = N; t >= 1; --t) {
    const int s0 = tree->stage_ptr[t], s1 = tree->stage_ptr[t + 1], m = s1 - s0;
    Phere.assign((size_t)m * mm, 0.0);
    const int nt = std::min(threads, m);
    std::vector<int> ok(nt, 1);
    auto work = [&](int tid) {
      NodeWork w{nu, ne, nv, cost->Wu, L.data(), Et.data()};
      w.init();
      std::vector<double> Phi(mm), K(mm), Mc((size_t)nu * std::max(1, ne), 0.0);
      std::vector<const double *> Pc;
      for (int v = s0 + tid; v < s1; v += nt) {
        Pc.clear();
        if (cend[v] > 0)
          for (int c = cbeg[v]; c < cend[v]; ++c) Pc.push_back(&Pbelow[(size_t)(c - below0) * mm]);
        const bool need_p = t > 1;
        if (!w.run(tree->prob[v], Pc.data(), (int)Pc.size(), Phi.data(), K.data(), Mc.data(),
                   need_p ? &Phere[(size_t)(v - s0) * mm] : nullptr)) {
          ok[tid] = 0;
          return;
        }
        sink(ctx, v, Phi.data(), K.data(), Mc.data());
      }
    };
    if (nt == 1) {
      work(0);
    } else {
      std::vector<std::thread> pool;
      for (int i = 0; i < nt; ++i) pool.emplace_back(work, i);
      for (auto &th : pool) th.join();
    }
    for (int i = 0; i < nt; ++i)
      if (!ok[i]) {
        set_error("per-node factor: L' Q L is not positive definite at stage %d (W_u not "
                  "positive definite on ker E, or a zero probability)", t);
        return RN_ERR_INVAL;
      }
    Pbelow.swap(Phere);
    below0 = s0;
  }
  return RN_OK;
}

}  // namespace rn

// Diagnostic export: the per-node matrices in FP64 on the host, no device
// work (include/rapidnet.h).
extern "C" int rapidnet_pernode_matrices(const rn_network *net, const rn_tree *tree,
                                         const rn_cost *cost, double *Phi, double *K,
                                         double *Mc) {
  rn::clear_error();
  if (!net || !tree || !cost || !Phi || !K) {
    rn::set_error("pernode_matrices: NULL argument");
    return RN_ERR_INVAL;
  }
  int rc = rn::pn_validate(net, tree, cost);
  if (rc) return rc;
  const int nu = net->nu, ne = net->ne, n = tree->n_nodes;
  const size_t mm = (size_t)nu * nu, me = (size_t)nu * ne;
  std::fill(Phi, Phi + mm, 0.0);
  std::fill(K, K + mm, 0.0);
  if (Mc && ne > 0) std::fill(Mc, Mc + me, 0.0);
  struct Out {
    double *Phi, *K, *Mc;
    size_t mm, me;
  } o{Phi, K, Mc, mm, me};
  auto sink = [](void *ctx, int v, const double *P, const double *Kv, const double *M) {
    Out *q = static_cast<Out *>(ctx);
    std::copy(P, P + q->mm, q->Phi + (size_t)v * q->mm);
    std::copy(Kv, Kv + q->mm, q->K + (size_t)v * q->mm);
    if (q->Mc && q->me) std::copy(M, M + q->me, q->Mc + (size_t)v * q->me);
  };
  (void)n;
  const int threads = (int)std::max(1u, std::thread::hardware_concurrency());
  return rn::pn_factor_host(net, tree, cost, threads, sink, &o, nullptr);
}
