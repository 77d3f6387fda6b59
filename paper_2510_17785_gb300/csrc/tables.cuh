// One-dimensional matrices of the Q_q Gauss-Lobatto basis and the (q+1)-point
// Gauss rule on [0,1], q = 1..8, in constant memory.  Every kernel indexes
// them with compile-time indices, so they are read as constant-bank operands.
//
//   B[q][g][a]  = l_a(x_g): basis a at Gauss point g         (interpolation)
//   D[q][g][h]  = l'_h(x_g) for the Lagrange basis on the Gauss points
//                 (collocation derivative at the Gauss points)
//   Bd[q][g][a] = l_a'(x_g): derivative of basis a at Gauss point g
//   E[qf][a][b] = l^{qc}_b(xi^{qf}_a), qc = qf/2 (p-prolongation, Section 3.1:
//                 the embedding V_{j,qc} -> V_{j,qf}; restriction is E^T)
//   EP[qf][a][b]: the same for the paper's level rule (qc = 2^k - 1 < qf)
//   gx[q][g], gw[q][g]: Gauss points and weights (used in FP64 setup kernels,
//                 read from global memory)
//
// Each translation unit holds its own copy (static __constant__) and uploads
// it through its own entry point.
#pragma once
#include <cuda_runtime.h>

#include "table_types.h"

namespace pmg {

static __constant__ Tables<double> c_tab_f64;
static __constant__ Tables<float> c_tab_f32;
// FP32 even and odd parts side by side, (Ee[k][q][i][j], Eo[k][q][i][j]), for packed two-lane FMAs
struct EOPacked {
  float2 v[4][PMG_MAXQ + 1][PMG_EOR][PMG_EOC];
};
static __constant__ EOPacked c_eo2_f32;
static __device__ Rules c_rules;          // set-up kernels only: global memory, not the constant bank

template <typename T>
__device__ __forceinline__ T tabB(int q, int g, int a);
template <>
__device__ __forceinline__ double tabB<double>(int q, int g, int a) { return c_tab_f64.B[q][g][a]; }
template <>
__device__ __forceinline__ float tabB<float>(int q, int g, int a) { return c_tab_f32.B[q][g][a]; }

template <typename T>
__device__ __forceinline__ T tabD(int q, int g, int h);
template <>
__device__ __forceinline__ double tabD<double>(int q, int g, int h) { return c_tab_f64.D[q][g][h]; }
template <>
__device__ __forceinline__ float tabD<float>(int q, int g, int h) { return c_tab_f32.D[q][g][h]; }

template <typename T>
__device__ __forceinline__ T tabE(int qf, int a, int b);
template <>
__device__ __forceinline__ double tabE<double>(int qf, int a, int b) { return c_tab_f64.E[qf][a][b]; }
template <>
__device__ __forceinline__ float tabE<float>(int qf, int a, int b) { return c_tab_f32.E[qf][a][b]; }

// prolongation for the paper's level rule: EP[qf][a][b] = l^{qc}_b(xi^{qf}_a),
// qc = the largest 2^k - 1 below qf (coarse_degree(qf, 1))
template <typename T>
__device__ __forceinline__ T tabEP(int qf, int a, int b);
template <>
__device__ __forceinline__ double tabEP<double>(int qf, int a, int b) { return c_tab_f64.EP[qf][a][b]; }
template <>
__device__ __forceinline__ float tabEP<float>(int qf, int a, int b) { return c_tab_f32.EP[qf][a][b]; }
// the prolongation table of level rule LR
template <typename T, int LR>
__device__ __forceinline__ T tabT(int qf, int a, int b) {
  if constexpr (LR == 1) return tabEP<T>(qf, a, b);
  else return tabE<T>(qf, a, b);
}

__device__ __forceinline__ float2 tabEO2(int k, int q, int i, int j) { return c_eo2_f32.v[k][q][i][j]; }

// even/odd parts of B, B^T, D, D^T (table_types.h)
template <typename T>
__device__ __forceinline__ T tabEe(int k, int q, int i, int j);
template <>
__device__ __forceinline__ double tabEe<double>(int k, int q, int i, int j) { return c_tab_f64.Ee[k][q][i][j]; }
template <>
__device__ __forceinline__ float tabEe<float>(int k, int q, int i, int j) { return c_tab_f32.Ee[k][q][i][j]; }
template <typename T>
__device__ __forceinline__ T tabEo(int k, int q, int i, int j);
template <>
__device__ __forceinline__ double tabEo<double>(int k, int q, int i, int j) { return c_tab_f64.Eo[k][q][i][j]; }
template <>
__device__ __forceinline__ float tabEo<float>(int k, int q, int i, int j) { return c_tab_f32.Eo[k][q][i][j]; }
template <typename T>
__device__ __forceinline__ T tabEm(int k, int q, int i);
template <>
__device__ __forceinline__ double tabEm<double>(int k, int q, int i) { return c_tab_f64.Em[k][q][i]; }
template <>
__device__ __forceinline__ float tabEm<float>(int k, int q, int i) { return c_tab_f32.Em[k][q][i]; }

static inline int upload_tables_tu(const Tables<double>& h64, const Tables<float>& h32, const Rules& r) {
  cudaError_t e = cudaMemcpyToSymbol(c_tab_f64, &h64, sizeof(h64));
  if (e != cudaSuccess) return (int)e;
  e = cudaMemcpyToSymbol(c_tab_f32, &h32, sizeof(h32));
  if (e != cudaSuccess) return (int)e;
  EOPacked pk;
  for (int k = 0; k < 4; ++k)
    for (int q = 0; q <= PMG_MAXQ; ++q)
      for (int i = 0; i < PMG_EOR; ++i)
        for (int j = 0; j < PMG_EOC; ++j) pk.v[k][q][i][j] = make_float2(h32.Ee[k][q][i][j], h32.Eo[k][q][i][j]);
  e = cudaMemcpyToSymbol(c_eo2_f32, &pk, sizeof(pk));
  if (e != cudaSuccess) return (int)e;
  return (int)cudaMemcpyToSymbol(c_rules, &r, sizeof(r));
}

}  // namespace pmg

// Every translation unit that includes this header registers its uploader
// when the library is loaded; upload_all_tables() (basis.cpp) calls them all
// for the current device.
namespace {
struct PmgTableRegistrar {
  PmgTableRegistrar() { pmg::register_table_uploader(&pmg::upload_tables_tu); }
};
static PmgTableRegistrar pmg_table_registrar;
}  // namespace
