// Layout of the one-dimensional tables (see tables.cuh for their meaning).
#pragma once

#define PMG_MAXQ 8

namespace pmg {

template <typename T>
struct Tables {
  T B[PMG_MAXQ + 1][PMG_MAXQ + 1][PMG_MAXQ + 1];
  T D[PMG_MAXQ + 1][PMG_MAXQ + 1][PMG_MAXQ + 1];
  T E[PMG_MAXQ + 1][PMG_MAXQ + 1][PMG_MAXQ + 1];
};

struct Rules {
  double gx[PMG_MAXQ + 1][PMG_MAXQ + 1];
  double gw[PMG_MAXQ + 1][PMG_MAXQ + 1];
  double Bd[PMG_MAXQ + 1][PMG_MAXQ + 1][PMG_MAXQ + 1];
  double Bg[PMG_MAXQ + 1][PMG_MAXQ + 2][PMG_MAXQ + 1];   // basis at the (q+2)-point rule
  double gx2[PMG_MAXQ + 1][PMG_MAXQ + 2];                 // (q+2)-point Gauss rule
  double gw2[PMG_MAXQ + 1][PMG_MAXQ + 2];
};

using TableUploader = int (*)(const Tables<double>&, const Tables<float>&, const Rules&);
// registry of the per-translation-unit uploaders (host code, basis.cpp)
void register_table_uploader(TableUploader f);
// upload the tables into every registered translation unit on the current
// device; returns 0 or the first CUDA error code
int upload_all_tables(const Tables<double>& t64, const Tables<float>& t32, const Rules& r);

}  // namespace pmg
