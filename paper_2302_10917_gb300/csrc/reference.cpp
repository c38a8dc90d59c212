// Reference-lattice tables of one refinement level (host set-up, run once per
// context). Sec. 3.2: W(K), V(K) are C0 piecewise P_p on the uniform m-fold
// subdivision of the reference triangle; M(F) is C0 piecewise P_p on the m
// sub-edges of a macro-edge. Every element matrix of the affine macro-element
// is a linear combination of the tables built here (element formation,
// Sec. 6.1), with coefficients from the element's Jacobian, kappa, tau and beta.
//
// The tables that involve Mh^-1 come from eliminating q = -grad u inside each
// macro-element: the q-rows of A_e read M q_x - Dx u + Fx u^ = 0, so
// q_x = M^-1 (Dx u - Fx u^); M^-1 D and M^-1 F scale with the affine map, so
// Dx^T M^-1 Dx etc. are fixed reference matrices times element scalars.
#include <cmath>
#include <stdexcept>
#include "internal.h"

namespace mehdg {
namespace {

// Gauss-Legendre nodes and weights on [0,1] by Newton iteration on P_n.
void gauss01(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      if (n == 1) { p0 = 1.0; p1 = z; }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      const double dz = p1 / dp;
      z -= dz;
      if (std::fabs(dz) < 1e-17) break;
    }
    {
      double p0 = 1.0, p1 = z;
      for (int k = 2; k <= n; ++k) {
        const double p2 = ((2.0 * k - 1.0) * z * p1 - (k - 1.0) * p0) / k;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
    }
    // roots come out in decreasing order of z; store ascending on [0,1]
    x[n - 1 - i] = 0.5 * (1.0 + z);
    w[n - 1 - i] = 1.0 / ((1.0 - z * z) * dp * dp);
  }
}

// P_p Lagrange basis of one triangle at barycentric point lam, multi-indices al.
// val[b], dl[b][k] = d phi_b / d lambda_k.
void lagrange_tri(int p, const std::vector<int>& al, int nloc, const double lam[3],
                  double* val, double (*dl)[3]) {
  for (int b = 0; b < nloc; ++b) {
    double f[3], df[3];
    for (int k = 0; k < 3; ++k) {
      double v = 1.0, d = 0.0;
      for (int j = 0; j < al[3 * b + k]; ++j) {
        const double g = (p * lam[k] - j) / (j + 1.0);
        d = d * g + v * (p / (j + 1.0));
        v *= g;
      }
      f[k] = v;
      df[k] = d;
    }
    val[b] = f[0] * f[1] * f[2];
    dl[b][0] = df[0] * f[1] * f[2];
    dl[b][1] = f[0] * df[1] * f[2];
    dl[b][2] = f[0] * f[1] * df[2];
  }
}

// Second derivatives of the same basis: h[b][k][l] = d^2 phi_b / d lambda_k d lambda_l.
void lagrange_tri_hess(int p, const std::vector<int>& al, int nloc, const double lam[3], double (*h)[3][3]) {
  for (int b = 0; b < nloc; ++b) {
    double f[3], df[3], ddf[3];
    for (int k = 0; k < 3; ++k) {
      double v = 1.0, d = 0.0, dd = 0.0;
      for (int j = 0; j < al[3 * b + k]; ++j) {
        const double g = (p * lam[k] - j) / (j + 1.0), gp = p / (j + 1.0);
        dd = dd * g + 2.0 * d * gp;
        d = d * g + v * gp;
        v *= g;
      }
      f[k] = v;
      df[k] = d;
      ddf[k] = dd;
    }
    for (int k = 0; k < 3; ++k)
      for (int l = 0; l < 3; ++l) {
        double v = 1.0;
        for (int t = 0; t < 3; ++t) {
          if (k == l) v *= (t == k ? ddf[t] : f[t]);
          else v *= (t == k || t == l) ? df[t] : f[t];
        }
        h[b][k][l] = v;
      }
  }
}

// 1D P_p Lagrange basis on [0,1] with equispaced nodes.
void lagrange_1d(int p, double s, double* out) {
  for (int k = 0; k <= p; ++k) {
    double v = 1.0;
    for (int j = 0; j <= p; ++j)
      if (j != k) v *= (s - double(j) / p) / (double(k - j) / p);
    out[k] = v;
  }
}

// In-place Cholesky A = L L^T (row-major n x n, lower triangle kept).
void cholesky(std::vector<double>& A, int n) {
  for (int j = 0; j < n; ++j) {
    double d = A[(size_t)j * n + j];
    for (int k = 0; k < j; ++k) d -= A[(size_t)j * n + k] * A[(size_t)j * n + k];
    if (!(d > 0.0)) throw std::runtime_error("reference mass matrix is not positive definite");
    d = std::sqrt(d);
    A[(size_t)j * n + j] = d;
    for (int i = j + 1; i < n; ++i) {
      double s = A[(size_t)i * n + j];
      for (int k = 0; k < j; ++k) s -= A[(size_t)i * n + k] * A[(size_t)j * n + k];
      A[(size_t)i * n + j] = s / d;
    }
  }
}

// X = A^-1 B for the Cholesky factor L of A (n x n), B row-major n x c.
std::vector<double> chol_solve(const std::vector<double>& L, int n, const std::vector<double>& B, int c) {
  std::vector<double> X(B);
  for (int col = 0; col < c; ++col) {
    for (int i = 0; i < n; ++i) {
      double s = X[(size_t)i * c + col];
      for (int k = 0; k < i; ++k) s -= L[(size_t)i * n + k] * X[(size_t)k * c + col];
      X[(size_t)i * c + col] = s / L[(size_t)i * n + i];
    }
    for (int i = n - 1; i >= 0; --i) {
      double s = X[(size_t)i * c + col];
      for (int k = i + 1; k < n; ++k) s -= L[(size_t)k * n + i] * X[(size_t)k * c + col];
      X[(size_t)i * c + col] = s / L[(size_t)i * n + i];
    }
  }
  return X;
}

// C = A^T B with A (r x a), B (r x b), row-major.
std::vector<double> atb(const std::vector<double>& A, int r, int a, const std::vector<double>& B, int b) {
  std::vector<double> C((size_t)a * b, 0.0);
  for (int k = 0; k < r; ++k)
    for (int i = 0; i < a; ++i) {
      const double aki = A[(size_t)k * a + i];
      if (aki == 0.0) continue;
      const double* brow = &B[(size_t)k * b];
      double* crow = &C[(size_t)i * b];
      for (int j = 0; j < b; ++j) crow[j] += aki * brow[j];
    }
  return C;
}

}  // namespace

void build_reference_tables(int m, int p, RefTables& T) {
  if (m < 1 || p < 1) throw std::runtime_error("m and p must be >= 1");
  T.m = m;
  T.p = p;
  T.P = m * p;
  T.P1 = T.P + 1;
  T.Q = (T.P + 1) * (T.P + 2) / 2;
  T.n_t = 3 * T.P1;
  const int P = T.P, P1 = T.P1, Q = T.Q, nt = T.n_t;
  auto node = [P](int a, int b) { return b * (P + 1) - b * (b - 1) / 2 + a; };

  // sub-triangles (published order) and their local P_p nodes
  T.subtri.clear();
  for (int sj = 0; sj < m; ++sj)
    for (int si = 0; si + sj <= m - 1; ++si) {
      int c[6] = {si, sj, si + 1, sj, si, sj + 1};
      T.subtri.insert(T.subtri.end(), c, c + 6);
    }
  for (int sj = 0; sj < m - 1; ++sj)
    for (int si = 0; si + sj <= m - 2; ++si) {
      int c[6] = {si + 1, sj + 1, si, sj + 1, si + 1, sj};
      T.subtri.insert(T.subtri.end(), c, c + 6);
    }
  T.nsub = (int)T.subtri.size() / 6;
  T.nloc = (p + 1) * (p + 2) / 2;
  std::vector<int> al;   // local multi-indices (A, B, C)
  for (int aC = 0; aC <= p; ++aC)
    for (int aB = 0; aB + aC <= p; ++aB) {
      al.push_back(p - aB - aC);
      al.push_back(aB);
      al.push_back(aC);
    }
  T.subnode.assign((size_t)T.nsub * T.nloc, 0);
  for (int s = 0; s < T.nsub; ++s) {
    const int* c = &T.subtri[6 * s];
    for (int b = 0; b < T.nloc; ++b) {
      const int a = al[3 * b] * c[0] + al[3 * b + 1] * c[2] + al[3 * b + 2] * c[4];
      const int bb = al[3 * b] * c[1] + al[3 * b + 1] * c[3] + al[3 * b + 2] * c[5];
      T.subnode[(size_t)s * T.nloc + b] = node(a, bb);
    }
  }
  // node -> (sub-triangle, local index) lists
  T.ns_ptr.assign(Q + 1, 0);
  for (int v : T.subnode) T.ns_ptr[v + 1]++;
  for (int i = 0; i < Q; ++i) T.ns_ptr[i + 1] += T.ns_ptr[i];
  T.ns_idx.assign(T.ns_ptr[Q], 0);
  {
    std::vector<int> fill(T.ns_ptr.begin(), T.ns_ptr.end() - 1);
    for (int s = 0; s < T.nsub; ++s)
      for (int b = 0; b < T.nloc; ++b) T.ns_idx[fill[T.subnode[(size_t)s * T.nloc + b]]++] = s * T.nloc + b;
  }

  // source / element rule on the unit triangle (collapsed Gauss, ng = p + 2)
  T.ng = p + 2;
  std::vector<double> gx, gw;
  gauss01(T.ng, gx, gw);
  T.uq = gx;
  T.nqs = T.ng * T.ng;
  T.wq.assign(T.nqs, 0.0);
  T.phiq.assign((size_t)T.nqs * T.nloc, 0.0);
  std::vector<double> dphi((size_t)T.nqs * T.nloc * 2);   // reference-sub-triangle gradients wrt (xi^, eta^)
  {
    std::vector<double> val(T.nloc);
    std::vector<double[3]> dl(T.nloc);
    for (int j = 0; j < T.ng; ++j)
      for (int i = 0; i < T.ng; ++i) {
        const int q = j * T.ng + i;
        const double xh = gx[i] * (1.0 - gx[j]), eh = gx[j];
        T.wq[q] = gw[i] * gw[j] * (1.0 - gx[j]);
        const double lam[3] = {1.0 - xh - eh, xh, eh};
        lagrange_tri(p, al, T.nloc, lam, val.data(), dl.data());
        for (int b = 0; b < T.nloc; ++b) {
          T.phiq[(size_t)q * T.nloc + b] = val[b];
          dphi[((size_t)q * T.nloc + b) * 2 + 0] = dl[b][1] - dl[b][0];   // d/dxi^ (lambda_B = xi^)
          dphi[((size_t)q * T.nloc + b) * 2 + 1] = dl[b][2] - dl[b][0];   // d/deta^ (lambda_C = eta^)
        }
      }
  }

  // mass and derivative matrices of the macro reference triangle
  T.Mh.assign((size_t)Q * Q, 0.0);
  T.Dxi.assign((size_t)Q * Q, 0.0);
  T.Deta.assign((size_t)Q * Q, 0.0);
  for (int s = 0; s < T.nsub; ++s) {
    const int* c = &T.subtri[6 * s];
    // sub-triangle map (xi, eta) = A + xi^ (B - A) + eta^ (C - A), all / m
    const double j00 = double(c[2] - c[0]) / m, j10 = double(c[3] - c[1]) / m;
    const double j01 = double(c[4] - c[0]) / m, j11 = double(c[5] - c[1]) / m;
    const double det = j00 * j11 - j01 * j10;
    // d(xi^, eta^)/d(xi, eta) = J_s^-1
    const double i00 = j11 / det, i01 = -j01 / det, i10 = -j10 / det, i11 = j00 / det;
    const int* nd = &T.subnode[(size_t)s * T.nloc];
    for (int q = 0; q < T.nqs; ++q) {
      const double w = T.wq[q] * std::fabs(det);
      for (int a = 0; a < T.nloc; ++a) {
        const double* da = &dphi[((size_t)q * T.nloc + a) * 2];
        const double dxi_a = da[0] * i00 + da[1] * i10;    // d phi / d xi
        const double deta_a = da[0] * i01 + da[1] * i11;   // d phi / d eta
        const double pa = T.phiq[(size_t)q * T.nloc + a];
        for (int b = 0; b < T.nloc; ++b) {
          const double pb = T.phiq[(size_t)q * T.nloc + b];
          const size_t ij = (size_t)nd[a] * Q + nd[b];
          T.Mh[ij] += w * pa * pb;
          T.Dxi[ij] += w * pb * dxi_a;
          T.Deta[ij] += w * pb * deta_a;
        }
      }
    }
  }

  // SUPG tables (Sec. 3.4): products of first derivatives and of first with
  // second derivatives of the lattice basis, sub-triangle by sub-triangle, and
  // the macro-reference gradients of every local basis function at the
  // source points
  T.Sxx.assign((size_t)Q * Q, 0.0);
  T.Syy.assign((size_t)Q * Q, 0.0);
  T.Ssym.assign((size_t)Q * Q, 0.0);
  for (auto* Lt : {&T.Lx_xx, &T.Lx_xy, &T.Lx_yy, &T.Ly_xx, &T.Ly_xy, &T.Ly_yy}) Lt->assign((size_t)Q * Q, 0.0);
  T.dphq.assign((size_t)T.nsub * T.nqs * T.nloc * 2, 0.0);
  {
    std::vector<double[3][3]> hl(T.nloc);
    std::vector<double> hq((size_t)T.nqs * T.nloc * 3);   // d2/dxi^2, d2/dxi^deta^, d2/deta^2 (local)
    for (int j = 0; j < T.ng; ++j)
      for (int i = 0; i < T.ng; ++i) {
        const int q = j * T.ng + i;
        const double xh = gx[i] * (1.0 - gx[j]), eh = gx[j];
        const double lam[3] = {1.0 - xh - eh, xh, eh};
        lagrange_tri_hess(p, al, T.nloc, lam, hl.data());
        const double u[3] = {-1.0, 1.0, 0.0}, v[3] = {-1.0, 0.0, 1.0};
        for (int b = 0; b < T.nloc; ++b) {
          double uu = 0.0, uv = 0.0, vv = 0.0;
          for (int k = 0; k < 3; ++k)
            for (int l = 0; l < 3; ++l) {
              uu += u[k] * hl[b][k][l] * u[l];
              uv += u[k] * hl[b][k][l] * v[l];
              vv += v[k] * hl[b][k][l] * v[l];
            }
          hq[((size_t)q * T.nloc + b) * 3 + 0] = uu;
          hq[((size_t)q * T.nloc + b) * 3 + 1] = uv;
          hq[((size_t)q * T.nloc + b) * 3 + 2] = vv;
        }
      }
    std::vector<double> gxi(T.nloc), geta(T.nloc), hxx(T.nloc), hxy(T.nloc), hyy(T.nloc);
    for (int s = 0; s < T.nsub; ++s) {
      const int* c = &T.subtri[6 * s];
      const double j00 = double(c[2] - c[0]) / m, j10 = double(c[3] - c[1]) / m;
      const double j01 = double(c[4] - c[0]) / m, j11 = double(c[5] - c[1]) / m;
      const double det = j00 * j11 - j01 * j10;
      const double i00 = j11 / det, i01 = -j01 / det, i10 = -j10 / det, i11 = j00 / det;
      const int* nd = &T.subnode[(size_t)s * T.nloc];
      for (int q = 0; q < T.nqs; ++q) {
        const double w = T.wq[q] * std::fabs(det);
        for (int a = 0; a < T.nloc; ++a) {
          const double* da = &dphi[((size_t)q * T.nloc + a) * 2];
          gxi[a] = da[0] * i00 + da[1] * i10;
          geta[a] = da[0] * i01 + da[1] * i11;
          const double* ha = &hq[((size_t)q * T.nloc + a) * 3];
          // (xi^, eta^) second derivatives to (xi, eta): c_xi = (i00, i10), c_eta = (i01, i11)
          hxx[a] = i00 * i00 * ha[0] + 2.0 * i00 * i10 * ha[1] + i10 * i10 * ha[2];
          hxy[a] = i00 * i01 * ha[0] + (i00 * i11 + i10 * i01) * ha[1] + i10 * i11 * ha[2];
          hyy[a] = i01 * i01 * ha[0] + 2.0 * i01 * i11 * ha[1] + i11 * i11 * ha[2];
          T.dphq[(((size_t)s * T.nqs + q) * T.nloc + a) * 2 + 0] = gxi[a];
          T.dphq[(((size_t)s * T.nqs + q) * T.nloc + a) * 2 + 1] = geta[a];
        }
        for (int a = 0; a < T.nloc; ++a)
          for (int b = 0; b < T.nloc; ++b) {
            const size_t ij = (size_t)nd[a] * Q + nd[b];
            T.Sxx[ij] += w * gxi[a] * gxi[b];
            T.Syy[ij] += w * geta[a] * geta[b];
            T.Ssym[ij] += w * (gxi[a] * geta[b] + geta[a] * gxi[b]);
            T.Lx_xx[ij] += w * gxi[a] * hxx[b];
            T.Lx_xy[ij] += w * gxi[a] * hxy[b];
            T.Lx_yy[ij] += w * gxi[a] * hyy[b];
            T.Ly_xx[ij] += w * geta[a] * hxx[b];
            T.Ly_xy[ij] += w * geta[a] * hxy[b];
            T.Ly_yy[ij] += w * geta[a] * hyy[b];
          }
      }
    }
  }

  // 1D trace mass Gh on [0,1] with m sub-intervals; boundary-data rule
  T.ngb = p + 2;
  gauss01(T.ngb, T.bu, T.bw);
  T.bpsi.assign((size_t)T.ngb * (p + 1), 0.0);
  for (int q = 0; q < T.ngb; ++q) lagrange_1d(p, T.bu[q], &T.bpsi[(size_t)q * (p + 1)]);
  T.Gh.assign((size_t)P1 * P1, 0.0);
  for (int s = 0; s < m; ++s)
    for (int q = 0; q < T.ngb; ++q)
      for (int r = 0; r <= p; ++r)
        for (int r2 = 0; r2 <= p; ++r2)
          T.Gh[(size_t)(s * p + r) * P1 + s * p + r2] +=
              T.bw[q] / m * T.bpsi[(size_t)q * (p + 1) + r] * T.bpsi[(size_t)q * (p + 1) + r2];
  {
    std::vector<double> L(T.Gh);
    cholesky(L, P1);
    std::vector<double> I((size_t)P1 * P1, 0.0);
    for (int i = 0; i < P1; ++i) I[(size_t)i * P1 + i] = 1.0;
    T.Ghinv = chol_solve(L, P1, I, P1);
  }

  // reference edge k runs from vertex k+1 to vertex k+2: lattice nodes along it
  T.enode.assign(3 * P1, 0);
  for (int t = 0; t <= P; ++t) {
    T.enode[0 * P1 + t] = node(P - t, t);   // (1,0) -> (0,1)
    T.enode[1 * P1 + t] = node(0, P - t);   // (0,1) -> (0,0)
    T.enode[2 * P1 + t] = node(t, 0);       // (0,0) -> (1,0)
  }
  // the restriction of the lattice basis to an edge is the trace basis, so
  // int_0^1 psi_t phi_i ds = Gh[t'][t] for i = enode[k][t'] (0 elsewhere)
  T.Fh.assign((size_t)Q * nt, 0.0);
  for (int k = 0; k < 3; ++k)
    for (int t2 = 0; t2 < P1; ++t2)
      for (int t = 0; t < P1; ++t)
        T.Fh[(size_t)T.enode[k * P1 + t2] * nt + k * P1 + t] = T.Gh[(size_t)t2 * P1 + t];

  // products through Mh^-1
  std::vector<double> L(T.Mh);
  cholesky(L, Q);
  T.Xxi = chol_solve(L, Q, T.Dxi, Q);
  T.Xeta = chol_solve(L, Q, T.Deta, Q);
  T.Yh = chol_solve(L, Q, T.Fh, nt);
  T.Kxx = atb(T.Dxi, Q, Q, T.Xxi, Q);
  T.Kyy = atb(T.Deta, Q, Q, T.Xeta, Q);
  {
    std::vector<double> a = atb(T.Dxi, Q, Q, T.Xeta, Q);
    std::vector<double> b = atb(T.Deta, Q, Q, T.Xxi, Q);
    T.Ksym.resize(a.size());
    for (size_t i = 0; i < a.size(); ++i) T.Ksym[i] = a[i] + b[i];
  }
  T.Pxi = atb(T.Dxi, Q, Q, T.Yh, nt);
  T.Peta = atb(T.Deta, Q, Q, T.Yh, nt);
  T.Hh = atb(T.Fh, Q, nt, T.Yh, nt);
  // column-major copies of the q-recovery tables (one thread per row reads them coalesced)
  T.XxiT.resize((size_t)Q * Q);
  T.XetaT.resize((size_t)Q * Q);
  T.YhT.resize((size_t)nt * Q);
  for (int i = 0; i < Q; ++i) {
    for (int j = 0; j < Q; ++j) {
      T.XxiT[(size_t)j * Q + i] = T.Xxi[(size_t)i * Q + j];
      T.XetaT[(size_t)j * Q + i] = T.Xeta[(size_t)i * Q + j];
    }
    for (int c = 0; c < nt; ++c) T.YhT[(size_t)c * Q + i] = T.Yh[(size_t)i * nt + c];
  }
}

}  // namespace mehdg

namespace mehdg {

// Trace tables of every face level R = 0 .. kMaxLevel (m = 2^R sub-intervals of
// [0,1]): the C0 P_p trace mass Gh_R and its inverse, and for r < R the
// transfer T_rR = Gh_r^-1 Pi^T Gh_R, Pi the level-r nodal basis at the
// level-R nodes. T_rR maps a level-R trace to the coefficients of its L2
// projection onto the level-r space, and the coarse side's face couplings
// to a level-R face are its own-level couplings times T_rR (the coarse
// basis restricted to the edge lies in the level-r trace space, Sec. 4.2).
void build_level_tables(int p, LevelTables& L) {
  L.p = p;
  std::vector<double> gx, gw;
  gauss01(p + 2, gx, gw);
  std::vector<double> psi((size_t)gx.size() * (p + 1));
  for (size_t q = 0; q < gx.size(); ++q) lagrange_1d(p, gx[q], &psi[q * (p + 1)]);
  std::vector<std::vector<double>> G(kMaxLevel + 1), Gi(kMaxLevel + 1);
  L.data.clear();
  for (int R = 0; R <= kMaxLevel; ++R) {
    const int m = 1 << R, n1 = m * p + 1;
    G[R].assign((size_t)n1 * n1, 0.0);
    for (int s = 0; s < m; ++s)
      for (size_t q = 0; q < gx.size(); ++q)
        for (int a = 0; a <= p; ++a)
          for (int b = 0; b <= p; ++b)
            G[R][(size_t)(s * p + a) * n1 + s * p + b] += gw[q] / m * psi[q * (p + 1) + a] * psi[q * (p + 1) + b];
    std::vector<double> Lc(G[R]);
    cholesky(Lc, n1);
    std::vector<double> I((size_t)n1 * n1, 0.0);
    for (int i = 0; i < n1; ++i) I[(size_t)i * n1 + i] = 1.0;
    Gi[R] = chol_solve(Lc, n1, I, n1);
    L.G_off[R] = (int64_t)L.data.size();
    L.data.insert(L.data.end(), G[R].begin(), G[R].end());
    L.Gi_off[R] = (int64_t)L.data.size();
    L.data.insert(L.data.end(), Gi[R].begin(), Gi[R].end());
  }
  for (int r = 0; r <= kMaxLevel; ++r)
    for (int R = 0; R <= kMaxLevel; ++R) {
      L.T_off[r][R] = -1;
      if (R <= r) continue;
      const int nc = (1 << r) * p + 1, nf = (1 << R) * p + 1;
      // Pi (nf x nc): level-r basis at the level-R nodes j / (nf - 1)
      std::vector<double> Pi((size_t)nf * nc, 0.0), v(p + 1);
      const int mc = 1 << r;
      for (int j = 0; j < nf; ++j) {
        const int num = j * mc, den = nf - 1;          // t = j / den, t * mc = num / den
        int s = num / den;
        if (s > mc - 1) s = mc - 1;
        const double loc = (double)(num - s * den) / den;
        lagrange_1d(p, loc, v.data());
        for (int a = 0; a <= p; ++a) Pi[(size_t)j * nc + s * p + a] = v[a];
      }
      // Pi^T G_R (nc x nf), then G_r^-1 (...)
      const std::vector<double> PtG = atb(Pi, nf, nc, G[R], nf);
      std::vector<double> T((size_t)nc * nf, 0.0);
      for (int i = 0; i < nc; ++i)
        for (int k = 0; k < nc; ++k) {
          const double g = Gi[r][(size_t)i * nc + k];
          for (int j = 0; j < nf; ++j) T[(size_t)i * nf + j] += g * PtG[(size_t)k * nf + j];
        }
      L.T_off[r][R] = (int64_t)L.data.size();
      L.data.insert(L.data.end(), T.begin(), T.end());
    }
}

}  // namespace mehdg
