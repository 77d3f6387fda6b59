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
    // prolongation from degree q/2 to q
    const int qc = q / 2;
    if (qc >= 1) {
      const std::vector<double> glc = gauss_lobatto(qc);
      const auto E = lagrange_matrix(glc, gl);   // [a][b]
      for (int a = 0; a <= q; ++a)
        for (int b = 0; b <= qc; ++b) t64.E[q][a][b] = E[a][b];
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
  for (int q = 0; q <= PMG_MAXQ; ++q)
    for (int i = 0; i <= PMG_MAXQ; ++i)
      for (int j = 0; j <= PMG_MAXQ; ++j) {
        t32.B[q][i][j] = (float)t64.B[q][i][j];
        t32.D[q][i][j] = (float)t64.D[q][i][j];
        t32.E[q][i][j] = (float)t64.E[q][i][j];
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

}  // namespace pmg
