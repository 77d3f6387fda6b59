// Internal (not part of the C ABI): a read-only view of one (mesh level,
// p-level) of a context, for entry points defined outside pmg_api.cu.
#pragma once
#include <stdint.h>

struct pmg_ctx;

namespace pmg {

struct LanczosView {
  int device = 0, dim = 0, N = 0, q = 0, ksteps = 0;
  int64_t npatch = 0;
  const double* G64 = nullptr;
  const double* dinv64 = nullptr;
  const float* G32 = nullptr;       // FP32 geometry, NULL if the context made none
  const float* dinv32 = nullptr;
  uint64_t seed = 0;
  double safety = 0.0, ratio = 0.0;
};

// PMG_OK, or PMG_ERR_ARG if the context is not set up or level/k are out of range
int lanczos_view(const pmg_ctx* ctx, int level, int k, LanczosView* v);
// records `msg` as the context's last error and returns `code`
int set_last_error(pmg_ctx* ctx, int code, const char* msg);

}  // namespace pmg
