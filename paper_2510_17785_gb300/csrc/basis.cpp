// Host-side 1D rules and tables (see basis.h).
#include "basis.h"

#include <cmath>
#include <cstring>

namespace pmg {

static void legendre(int n, double x, double& P, double& dP) {
  // P_n and P_n' by the three-term recurrence
  double p0 = 1.0, p1 = x;
  if (n == 0) { P = 1.0; dP = 0.0; return; }
  for (int k = 1; k < n; ++k) {
    const double p2 = ((2.0 * k + 1.0) * x * p1 - k * p0) / (k + 1.0);
    p0 = p1;
    p1 = p2;
  }
  P = p1;
  dP = n * (x * p1 - p0) / (x * x - 1.0);
}

void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < n; ++i) {
    double z = std::cos(M_PI * (i + 0.75) / (n + 0.5));
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(n, z, P, dP);
      const double dz = P / dP;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    double P, dP;
    legendre(n, z, P, dP);
    // ascending order on [0, 1]
    x[n - 1 - i] = 0.5 * (z + 1.0);
    w[n - 1 - i] = 0.5 * 2.0 / ((1.0 - z * z) * dP * dP);
  }
}

std::vector<double> gauss_lobatto(int q) {
  std::vector<double> x(q + 1);
  x[0] = 0.0;
  x[q] = 1.0;
  for (int i = 1; i < q; ++i) {
    double z = -std::cos(M_PI * i / q);   // Chebyshev-Gauss-Lobatto guess, ascending
    for (int it = 0; it < 100; ++it) {
      double P, dP;
      legendre(q, z, P, dP);
      const double d2P = (2.0 * z * dP - q * (q + 1.0) * P) / (1.0 - z * z);
      const double dz = dP / d2P;
      z -= dz;
      if (std::fabs(dz) < 1e-16) break;
    }
    x[i] = 0.5 * (z + 1.0);
  }
  return x;
}

static std::vector<double> bary_weights(const std::vector<double>& nodes) {
  const int n = (int)nodes.size();
  std::vector<double> w(n, 1.0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k)
      if (k != j) w[j] /= (nodes[j] - nodes[k]);
  return w;
}

std::vector<std::vector<double>> lagrange_matrix(const std::vector<double>& nodes, const std::vector<double>& x) {
  const int n = (int)nodes.size();
  const std::vector<double> w = bary_weights(nodes);
  std::vector<std::vector<double>> L(x.size(), std::vector<double>(n, 0.0));
  for (size_t i = 0; i < x.size(); ++i) {
    int hit = -1;
    for (int j = 0; j < n; ++j)
      if (x[i] == nodes[j]) hit = j;
    if (hit >= 0) {
      L[i][hit] = 1.0;
      continue;
    }
    double den = 0.0;
    for (int j = 0; j < n; ++j) den += w[j] / (x[i] - nodes[j]);
    for (int j = 0; j < n; ++j) L[i][j] = (w[j] / (x[i] - nodes[j])) / den;
  }
  return L;
}

std::vector<std::vector<double>> diff_matrix(const std::vector<double>& nodes) {
  const int n = (int)nodes.size();
  const std::vector<double> w = bary_weights(nodes);
  std::vector<std::vector<double>> D(n, std::vector<double>(n, 0.0));
  for (int i = 0; i < n; ++i) {
    double s = 0.0;
    for (int j = 0; j < n; ++j) {
      if (j == i) continue;
      D[i][j] = (w[j] / w[i]) / (nodes[i] - nodes[j]);
      s += D[i][j];
    }
    D[i][i] = -s;
  }
  return D;
}

void build_tables(Tables<double>& t64, Tables<float>& t32, Rules& r) {
  std::memset(&t64, 0, sizeof(t64));
  std::memset(&t32, 0, sizeof(t32));
  std::memset(&r, 0, sizeof(r));
  for (int q = 1; q <= PMG_MAXQ; ++q) {
    const int n = q + 1;
    std::vector<double> gx, gw;
    gauss_rule(n, gx, gw);
    const std::vector<double> gl = gauss_lobatto(q);
    const auto B = lagrange_matrix(gl, gx);     // [g][a]
    const auto D = diff_matrix(gx);             // [g][h]
    for (int a = 0; a < n; ++a) r.gll[q][a] = gl[a];
    for (int g = 0; g < n; ++g) {
      r.gx[q][g] = gx[g];
      r.gw[q][g] = gw[g];
      for (int a = 0; a < n; ++a) {
        t64.B[q][g][a] = B[g][a];
        t64.D[q][g][a] = D[g][a];
        double bd = 0.0;
        for (int h = 0; h < n; ++h) bd += D[g][h] * B[h][a];
        r.Bd[q][g][a] = bd;
      }
    }
    // prolongation from degree q/2 to q, and from the paper rule's coarse degree
    for (int rule = 0; rule < 2; ++rule) {
      const int qc = coarse_degree(q, rule);
      if (qc < 1) continue;
      const std::vector<double> glc = gauss_lobatto(qc);
      const auto E = lagrange_matrix(glc, gl);   // [a][b]
      for (int a = 0; a <= q; ++a)
        for (int b = 0; b <= qc; ++b) (rule == 0 ? t64.E : t64.EP)[q][a][b] = E[a][b];
    }
    // (q+2)-point rule for load vectors
    std::vector<double> gx2, gw2;
    gauss_rule(q + 2, gx2, gw2);
    const auto B2 = lagrange_matrix(gl, gx2);
    for (int g = 0; g < q + 2; ++g) {
      r.gx2[q][g] = gx2[g];
      r.gw2[q][g] = gw2[g];
      for (int a = 0; a <= q; ++a) r.Bg[q][g][a] = B2[g][a];
    }
  }
  // even/odd parts of B, B^T, D, D^T (see table_types.h); M is first made
  // exactly (anti)symmetric by averaging M[i][j] with S M[n-1-i][n-1-j]
  for (int q = 1; q <= PMG_MAXQ; ++q) {
    const int n = q + 1, h = n / 2;
    for (int k = 0; k < 4; ++k) {
      const double S = (k == EO_D || k == EO_DT) ? -1.0 : 1.0;
      auto raw = [&](int i, int j) {
        switch (k) {
          case EO_B: return t64.B[q][i][j];
          case EO_BT: return t64.B[q][j][i];
          case EO_D: return t64.D[q][i][j];
          default: return t64.D[q][j][i];
        }
      };
      auto M = [&](int i, int j) { return 0.5 * (raw(i, j) + S * raw(n - 1 - i, n - 1 - j)); };
      for (int i = 0; i <= h && i < n; ++i) {
        for (int j = 0; j < h; ++j) {
          t64.Ee[k][q][i][j] = 0.5 * (M(i, j) + M(i, n - 1 - j));
          t64.Eo[k][q][i][j] = 0.5 * (M(i, j) - M(i, n - 1 - j));
        }
        t64.Em[k][q][i] = (n % 2 == 1) ? M(i, h) : 0.0;
      }
    }
  }
  for (int q = 0; q <= PMG_MAXQ; ++q) {
    for (int i = 0; i <= PMG_MAXQ; ++i)
      for (int j = 0; j <= PMG_MAXQ; ++j) {
        t32.B[q][i][j] = (float)t64.B[q][i][j];
        t32.D[q][i][j] = (float)t64.D[q][i][j];
        t32.E[q][i][j] = (float)t64.E[q][i][j];
        t32.EP[q][i][j] = (float)t64.EP[q][i][j];
      }
    for (int k = 0; k < 4; ++k)
      for (int i = 0; i < PMG_EOR; ++i) {
        t32.Em[k][q][i] = (float)t64.Em[k][q][i];
        for (int j = 0; j < PMG_EOC; ++j) {
          t32.Ee[k][q][i][j] = (float)t64.Ee[k][q][i][j];
          t32.Eo[k][q][i][j] = (float)t64.Eo[k][q][i][j];
        }
      }
  }
}

void h_prolongation_band(int q, int Nc, std::vector<double>& W, std::vector<int>& start) {
  const int Nf = 2 * Nc;
  const int Mf = q * Nf + 1;
  const std::vector<double> gl = gauss_lobatto(q);
  W.assign((size_t)Mf * (q + 1), 0.0);
  start.assign(Mf, 0);
  for (int K = 0; K < Mf; ++K) {
    int cf = K / q;
    if (cf > Nf - 1) cf = Nf - 1;
    const int a = K - q * cf;
    const int cc = cf / 2, child = cf % 2;
    const double xi = 0.5 * (child + gl[a]);
    const auto L = lagrange_matrix(gl, std::vector<double>{xi});
    start[K] = q * cc;
    for (int b = 0; b <= q; ++b) W[(size_t)K * (q + 1) + b] = L[0][b];
  }
}

void h_restriction_band(int q, int Nc, std::vector<double>& W, std::vector<int>& start, int& width) {
  std::vector<double> Pw;
  std::vector<int> Ps;
  h_prolongation_band(q, Nc, Pw, Ps);
  const int Mf = 2 * q * Nc + 1, Mc = q * Nc + 1;
  width = 4 * q + 1;
  W.assign((size_t)Mc * width, 0.0);
  start.assign(Mc, 0);
  for (int J = 0; J < Mc; ++J) start[J] = 2 * J - 2 * q;
  for (int K = 0; K < Mf; ++K)
    for (int b = 0; b <= q; ++b) {
      const int J = Ps[K] + b;
      const int t = K - start[J];
      if (t >= 0 && t < width) W[(size_t)J * width + t] += Pw[(size_t)K * (q + 1) + b];
    }
}

static std::vector<TableUploader>& uploaders() {
  static std::vector<TableUploader> v;
  return v;
}

void register_table_uploader(TableUploader f) { uploaders().push_back(f); }

int upload_all_tables(const Tables<double>& t64, const Tables<float>& t32, const Rules& r) {
  for (TableUploader f : uploaders()) {
    const int e = f(t64, t32, r);
    if (e != 0) return e;
  }
  return 0;
}



// ---- fast diagonalisation of the reference Cartesian patch ------------------
// 1D stiffness K and mass M of the degree-q basis on two unit cells, restricted
// to the 2q-1 interior nodes (Gauss rule with q+1 points per cell, exact for
// these polynomial products).  The generalised eigenproblem K s = lambda M s is
// reduced with the Cholesky factor of M (M = L L^T, C = L^-1 K L^-T) and C is
// diagonalised by cyclic Jacobi rotations; S = L^-T Q then satisfies
// S^T M S = I and S^T K S = diag(lambda), so the d-dimensional reference
// operator K(x)M(x)M + M(x)K(x)M + M(x)M(x)K has the inverse
// (S(x)S(x)S) diag(1 / (lambda_i + lambda_j + lambda_k)) (S(x)S(x)S)^T.
std::vector<double> fdm_table(int q) {
  const int n = q + 1, mi = 2 * q - 1;
  std::vector<double> gx, gw;
  gauss_rule(n, gx, gw);
  const std::vector<double> gl = gauss_lobatto(q);
  const auto B = lagrange_matrix(gl, gx);     // [g][a]
  const auto Dg = diff_matrix(gx);            // [g][h]
  std::vector<std::vector<double>> Bd(n, std::vector<double>(n, 0.0));
  for (int g = 0; g < n; ++g)
    for (int a = 0; a < n; ++a)
      for (int h = 0; h < n; ++h) Bd[g][a] += Dg[g][h] * B[h][a];
  std::vector<double> K((size_t)mi * mi, 0.0), M((size_t)mi * mi, 0.0);
  for (int c = 0; c < 2; ++c)
    for (int a = 0; a <= q; ++a)
      for (int b = 0; b <= q; ++b) {
        const int i = c * q + a - 1, j = c * q + b - 1;        // interior index, -1 / mi: boundary
        if (i < 0 || j < 0 || i >= mi || j >= mi) continue;
        double k = 0.0, m = 0.0;
        for (int g = 0; g < n; ++g) {
          k += gw[g] * Bd[g][a] * Bd[g][b];
          m += gw[g] * B[g][a] * B[g][b];
        }
        K[(size_t)i * mi + j] += k;
        M[(size_t)i * mi + j] += m;
      }
  // M = L L^T
  std::vector<double> L((size_t)mi * mi, 0.0);
  for (int j = 0; j < mi; ++j) {
    double d = M[(size_t)j * mi + j];
    for (int k = 0; k < j; ++k) d -= L[(size_t)j * mi + k] * L[(size_t)j * mi + k];
    d = std::sqrt(d);
    L[(size_t)j * mi + j] = d;
    for (int i = j + 1; i < mi; ++i) {
      double v = M[(size_t)i * mi + j];
      for (int k = 0; k < j; ++k) v -= L[(size_t)i * mi + k] * L[(size_t)j * mi + k];
      L[(size_t)i * mi + j] = v / d;
    }
  }
  // Li = L^-1 (lower triangular)
  std::vector<double> Li((size_t)mi * mi, 0.0);
  for (int c = 0; c < mi; ++c)
    for (int i = 0; i < mi; ++i) {
      double v = (i == c) ? 1.0 : 0.0;
      for (int k = 0; k < i; ++k) v -= L[(size_t)i * mi + k] * Li[(size_t)k * mi + c];
      Li[(size_t)i * mi + c] = v / L[(size_t)i * mi + i];
    }
  // C = Li K Li^T
  std::vector<double> T((size_t)mi * mi, 0.0), C((size_t)mi * mi, 0.0);
  for (int i = 0; i < mi; ++i)
    for (int j = 0; j < mi; ++j)
      for (int k = 0; k < mi; ++k) T[(size_t)i * mi + j] += Li[(size_t)i * mi + k] * K[(size_t)k * mi + j];
  for (int i = 0; i < mi; ++i)
    for (int j = 0; j < mi; ++j)
      for (int k = 0; k < mi; ++k) C[(size_t)i * mi + j] += T[(size_t)i * mi + k] * Li[(size_t)j * mi + k];
  // cyclic Jacobi: C = Q diag Q^T
  std::vector<double> Q((size_t)mi * mi, 0.0);
  for (int i = 0; i < mi; ++i) Q[(size_t)i * mi + i] = 1.0;
  for (int sweep = 0; sweep < 100; ++sweep) {
    double off = 0.0;
    for (int i = 0; i < mi; ++i)
      for (int j = i + 1; j < mi; ++j) off += C[(size_t)i * mi + j] * C[(size_t)i * mi + j];
    if (off < 1e-30) break;
    for (int p = 0; p < mi; ++p)
      for (int r = p + 1; r < mi; ++r) {
        const double apr = C[(size_t)p * mi + r];
        if (std::fabs(apr) < 1e-300) continue;
        const double app = C[(size_t)p * mi + p], arr = C[(size_t)r * mi + r];
        const double tau = (arr - app) / (2.0 * apr);
        const double t = (tau >= 0 ? 1.0 : -1.0) / (std::fabs(tau) + std::sqrt(1.0 + tau * tau));
        const double cs = 1.0 / std::sqrt(1.0 + t * t), sn = t * cs;
        for (int k = 0; k < mi; ++k) {            // C <- J^T C J
          const double ckp = C[(size_t)k * mi + p], ckr = C[(size_t)k * mi + r];
          C[(size_t)k * mi + p] = cs * ckp - sn * ckr;
          C[(size_t)k * mi + r] = sn * ckp + cs * ckr;
        }
        for (int k = 0; k < mi; ++k) {
          const double cpk = C[(size_t)p * mi + k], crk = C[(size_t)r * mi + k];
          C[(size_t)p * mi + k] = cs * cpk - sn * crk;
          C[(size_t)r * mi + k] = sn * cpk + cs * crk;
        }
        for (int k = 0; k < mi; ++k) {            // Q <- Q J
          const double qkp = Q[(size_t)k * mi + p], qkr = Q[(size_t)k * mi + r];
          Q[(size_t)k * mi + p] = cs * qkp - sn * qkr;
          Q[(size_t)k * mi + r] = sn * qkp + cs * qkr;
        }
      }
  }
  // S = Li^T Q; output [S (row i: node, column k: mode)][lambda][diag K][diag M]
  std::vector<double> out((size_t)mi * mi + 3 * mi, 0.0);
  for (int i = 0; i < mi; ++i)
    for (int k = 0; k < mi; ++k) {
      double v = 0.0;
      for (int j = 0; j < mi; ++j) v += Li[(size_t)j * mi + i] * Q[(size_t)j * mi + k];
      out[(size_t)i * mi + k] = v;
    }
  for (int k = 0; k < mi; ++k) {
    out[(size_t)mi * mi + k] = C[(size_t)k * mi + k];
    out[(size_t)mi * mi + mi + k] = K[(size_t)k * mi + k];
    out[(size_t)mi * mi + 2 * mi + k] = M[(size_t)k * mi + k];
  }
  return out;
}

}  // namespace pmg
