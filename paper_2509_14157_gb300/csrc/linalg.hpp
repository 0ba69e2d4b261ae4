// Small dense host linear algebra (k <= a few hundred): the Davidson subspace
// eigenproblem and DIIS linear systems. These are O(k^3) with k the subspace
// size; all vector-length work stays on the device.
#pragma once
#include <complex>
#include <vector>

namespace fnocc {

// Eigenvalues w[n] and right eigenvectors (column j of V, V[i*n+j]) of a real
// non-symmetric n x n row-major matrix A. Complex arithmetic throughout:
// Householder reduction to Hessenberg form, shifted QR (Wilkinson shifts,
// Givens rotations, deflation), eigenvectors by inverse iteration on A.
void eig_nonsym(int n, const std::vector<double> &A, std::vector<std::complex<double>> &w,
                std::vector<std::complex<double>> &V);

// Solves A x = b (n x n, row-major) by Gaussian elimination with partial
// pivoting. Returns false if A is numerically singular.
bool solve_linear(int n, std::vector<double> A, std::vector<double> b, std::vector<double> &x);

}  // namespace fnocc
