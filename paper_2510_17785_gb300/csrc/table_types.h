// Layout of the one-dimensional tables (see tables.cuh for their meaning).
#pragma once
#include <cuda_runtime.h>

#define PMG_MAXQ 8

namespace pmg {

// Even/odd parts of the n x n (n = q + 1) one-dimensional matrices M with
// M[n-1-i][n-1-j] = S M[i][j]: the interpolation B and its transpose (S = +1;
// Gauss points and Gauss-Lobatto nodes are symmetric about 1/2) and the
// collocation derivative D and its transpose (S = -1).  With h = n / 2,
//   Ee[i][j] = (M[i][j] + M[i][n-1-j]) / 2,  Eo[i][j] = (M[i][j] - M[i][n-1-j]) / 2  (j < h),
//   Em[i]    = M[i][h] (n odd),
// for rows i <= h; y = M x then follows from the even and odd parts of x
// (sf.cuh, eo_apply).
#define PMG_EOR (PMG_MAXQ / 2 + 1)       // rows i = 0 .. h (h <= 4 for n <= 9)
#define PMG_EOC ((PMG_MAXQ + 1) / 2)     // columns j < h
enum { EO_B = 0, EO_BT = 1, EO_D = 2, EO_DT = 3 };

// p-level sequences of the local V-cycle (Section 3.1): rule 0 halves the
// degree (p, p/2, ..., 1); rule 1 is the paper's nested sequence 1, 3, 7,
// 15, ... below p with p on top (p = 8: 8, 7, 3, 1)
__host__ __device__ constexpr int coarse_degree(int q, int rule) {
  if (q <= 1) return 0;
  if (rule == 0) return q / 2;
  int c = 1;
  while (2 * c + 1 < q) c = 2 * c + 1;
  return c;
}
__host__ __device__ constexpr int level_degree(int p, int rule, int k) {
  return k == 0 ? p : coarse_degree(level_degree(p, rule, k - 1), rule);
}
__host__ __device__ constexpr int nlevels_rule(int p, int rule) {
  return p <= 1 ? 1 : 1 + nlevels_rule(coarse_degree(p, rule), rule);
}
// the two rules give different sequences for degree p
__host__ __device__ constexpr bool rules_differ(int p) {
  for (int k = 0; k < 8; ++k)
    if (level_degree(p, 0, k) != level_degree(p, 1, k)) return true;
  return false;
}

template <typename T>
struct Tables {
  T B[PMG_MAXQ + 1][PMG_MAXQ + 1][PMG_MAXQ + 1];
  T D[PMG_MAXQ + 1][PMG_MAXQ + 1][PMG_MAXQ + 1];
  T E[PMG_MAXQ + 1][PMG_MAXQ + 1][PMG_MAXQ + 1];
  T EP[PMG_MAXQ + 1][PMG_MAXQ + 1][PMG_MAXQ + 1];
  T Ee[4][PMG_MAXQ + 1][PMG_EOR][PMG_EOC];
  T Eo[4][PMG_MAXQ + 1][PMG_EOR][PMG_EOC];
  T Em[4][PMG_MAXQ + 1][PMG_EOR];
};

struct Rules {
  double gx[PMG_MAXQ + 1][PMG_MAXQ + 1];
  double gw[PMG_MAXQ + 1][PMG_MAXQ + 1];
  double Bd[PMG_MAXQ + 1][PMG_MAXQ + 1][PMG_MAXQ + 1];
  double Bg[PMG_MAXQ + 1][PMG_MAXQ + 2][PMG_MAXQ + 1];   // basis at the (q+2)-point rule
  double gx2[PMG_MAXQ + 1][PMG_MAXQ + 2];                 // (q+2)-point Gauss rule
  double gw2[PMG_MAXQ + 1][PMG_MAXQ + 2];
  double gll[PMG_MAXQ + 1][PMG_MAXQ + 1];                 // Gauss-Lobatto nodes on [0, 1]
};

using TableUploader = int (*)(const Tables<double>&, const Tables<float>&, const Rules&);
// registry of the per-translation-unit uploaders (host code, basis.cpp)
void register_table_uploader(TableUploader f);
// upload the tables into every registered translation unit on the current
// device; returns 0 or the first CUDA error code
int upload_all_tables(const Tables<double>& t64, const Tables<float>& t32, const Rules& r);

}  // namespace pmg
