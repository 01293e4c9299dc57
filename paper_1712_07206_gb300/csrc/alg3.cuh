// The operand product of the paper's Alg. 3 (Sec. 5.1): its zgemm/zhemm steps
//   X_a = T^BA A_a + T^BB B_a / 2,   Y_a = T^AA A_a
// are the rows of M [A_a; B_a] with the 2N_L x 2N_L matrix
//   M = [[T^BA, T^BB / 2], [T^AA, 0]]   (rows r < N_L: X, rows N_L + i: Y_i),
// and its zher2k + zherkx H = X^H B + B^H X + A^H Y is the contraction L^H R
// of L_a = [X_a; B_a; A_a] and R_a = [B_a; X_a; Y_a] (3 N_L rows per atom):
// row r of M [A_a; B_a] is column N_L + r of R_a and, for r < N_L, column r
// of L_a.
//
// The paper's Alg. 1 differs only in the H_AA part: where the Cholesky
// factorisation T^AA = C C^H succeeds it forms Z_a = C^H A_a and adds
// Z_a^H Z_a (zherk), elsewhere A_a^H (T^AA A_a) (zgemm).  In the stacked form
// the Y rows of M become C^H (upper triangular) for such a slot, and the third
// block of L_a is then Y_a as well: L_a = [X_a; B_a; Y_a], R_a = [B_a; X_a; Y_a].
#pragma once

#include <cstdint>

namespace flapw {
namespace alg3 {

// Element (i, j) of a Hermitian T block given by its lower triangle (row-major).
__device__ __forceinline__ double2 t_elem(const double2* T, int n, int i, int j) {
  if (i >= j) return T[(int64_t)i * n + j];
  const double2 v = T[(int64_t)j * n + i];
  return make_double2(v.x, -v.y);
}

// M(r, c) for one T block (n = 2 N_L).
__device__ __forceinline__ double2 m_elem(const double2* T, int n, int nL, int r, int c) {
  if (r < nL) {
    const double2 v = t_elem(T, n, nL + r, c);
    return (c < nL) ? v : make_double2(0.5 * v.x, 0.5 * v.y);
  }
  return (c < nL) ? t_elem(T, n, r - nL, c) : make_double2(0.0, 0.0);
}

}  // namespace alg3
}  // namespace flapw
