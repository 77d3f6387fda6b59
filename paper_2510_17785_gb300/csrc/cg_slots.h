// Fixed sizes of the deterministic dot products and the slots of the CG
// scalars kept in device memory.
#pragma once

namespace pmg {

constexpr int DOT_BLOCKS = 608;     // 4 x 152 SMs; fixed, so the summation order is fixed
constexpr int DOT_THREADS = 256;

enum { S_RZ = 0, S_RZ_OLD, S_PAP, S_RR, S_ALPHA, S_BETA, S_NSLOT };

}  // namespace pmg
