// One row of the matrix-free operators (Sec. 3.1: the pressure Poisson
// matrix; the backward-Euler velocity matrices of the diffusion substep),
// shared by the persistent solvers and the graph-form solve.  Internal.
//
// Inputs: the centre value xc and the six neighbour values, where a
// neighbour outside the array holds xc (the callers substitute it); the row
// overrides the wall neighbours by its own rule:
//   pressure   Neumann: the missing neighbour equals xc (row n_c xc - sum);
//   velocity   comp = kind - 1; faces normal to a wall of their own axis are
//              known zeros (row 0); along the other axes a missing
//              neighbour is the ghost -xc (wall value 0 mirrored), and the
//              row is xc + c (6 xc - sum).
#pragma once

#include "cfd_internal.h"

namespace cfd {

template <typename T>
__device__ __forceinline__ T stencil_row(int kind, T c, int i, int j, int k, int mx, int my, int mz, T xc,
                                         T xm, T xp, T ym, T yp, T zm, T zp) {
  if (kind == kOpPressure) {
    if (i == 0) xm = xc;
    if (i == mx - 1) xp = xc;
    if (j == 0) ym = xc;
    if (j == my - 1) yp = xc;
    if (k == 0) zm = xc;
    if (k == mz - 1) zp = xc;
    return fma(T(6), xc, -(((((xm + xp) + ym) + yp) + zm) + zp));
  }
  const int comp = kind - 1;
  const bool wall_row = (comp == 0) ? (i == 0 || i == mx - 1)
                                    : (comp == 1) ? (j == 0 || j == my - 1) : (k == 0 || k == mz - 1);
  if (wall_row) return T(0);
  const T g = -xc;
  if (comp != 0) {
    if (i == 0) xm = g;
    if (i == mx - 1) xp = g;
  }
  if (comp != 1) {
    if (j == 0) ym = g;
    if (j == my - 1) yp = g;
  }
  if (comp != 2) {
    if (k == 0) zm = g;
    if (k == mz - 1) zp = g;
  }
  const T lap = fma(T(6), xc, -(((((xm + xp) + ym) + yp) + zm) + zp));
  return fma(c, lap, xc);
}

}  // namespace cfd
