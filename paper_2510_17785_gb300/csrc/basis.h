// Host-side 1D rules and the tables uploaded to constant memory.
//
// Gauss nodes are the roots of the Legendre polynomial P_n found by Newton
// iteration from Chebyshev initial guesses, weights 2 / ((1 - x^2) P_n'(x)^2);
// Gauss-Lobatto nodes are the endpoints and the roots of P_q', found by
// Newton iteration on P_q' using the Legendre differential equation for P_q''.
// Lagrange bases are evaluated with the barycentric formula, the collocation
// derivative with the barycentric differentiation matrix (Berrut & Trefethen,
// "Barycentric Lagrange interpolation", SIAM Review 2004).  All rules are
// mapped to [0, 1].
#pragma once
#include <vector>

#include "table_types.h"

namespace pmg {

void gauss_rule(int n, std::vector<double>& x, std::vector<double>& w);
std::vector<double> gauss_lobatto(int q);
// L[i][j] = l_j(x_i) for the Lagrange basis on `nodes`
std::vector<std::vector<double>> lagrange_matrix(const std::vector<double>& nodes, const std::vector<double>& x);
// D[i][j] = l_j'(nodes_i) (differentiation matrix on the nodes)
std::vector<std::vector<double>> diff_matrix(const std::vector<double>& nodes);

void build_tables(Tables<double>& t64, Tables<float>& t32, Rules& r);

// 1D h-prolongation from a mesh of Nc cells to one of 2 Nc cells at degree q,
// as a band: row K (fine node) has width q+1 starting at column start[K].
void h_prolongation_band(int q, int Nc, std::vector<double>& W, std::vector<int>& start);
// its transpose as a band of width 4q+1 (start may be negative)
void h_restriction_band(int q, int Nc, std::vector<double>& W, std::vector<int>& start, int& width);

// Fast-diagonalisation table of the reference Cartesian patch at degree q
// (Section 3.1, Cartesian-reinforced smoother), mi = 2q - 1 interior nodes:
// [S: mi x mi row-major, S^T M S = I, S^T K S = diag(lambda)][lambda: mi]
// [diag K: mi][diag M: mi] for the 1D stiffness K and mass M on two unit cells.
std::vector<double> fdm_table(int q);

}  // namespace pmg
