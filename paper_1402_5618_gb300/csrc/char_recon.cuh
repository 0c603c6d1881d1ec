// char_recon.cuh -- the characteristic-wise compact-WENO reconstruction of
// one sweep direction (Sec. 2.3, steps 1-4, eqs. (cha-1), (1DEuler-FVC)).
//
// For every line and each side (minus: U^-_{i+1/2}, plus: U^+_{i-1/2}) the
// block tridiagonal system of the line is assembled and solved by one
// thread, walking the line in the stable elimination order (minus left to
// right, plus right to left).  At each position the thread forms the Roe
// average of the two cells adjacent to the unknown's face, its left
// eigenvectors l^(k) (eq. (leigenv); the 4 x 4 system with the shear field in
// 2-D), the characteristic variables l^(k) ubar of the five-cell stencil, the
// WENO-Z weights of each field and the block row diag(a, b, c) L; the block
// Thomas multipliers go to a scratch buffer laid out [row][entry][line] so
// that the threads of a warp (consecutive lines) access it together.
// Periodic lines carry the Woodbury columns of the cyclic correction through
// the same pass.  Bounded lines close the first and last unknown with the
// explicit WENO5-Z value of each characteristic variable at that face.
//
// The output planes hold U^- and U^+ of every cell in the state's layout and
// grid variable order; the line kernel limits them, evaluates the face
// fluxes and forms the stage update.
#pragma once

#include <cuda_runtime.h>

namespace ppk {

struct CharArgs {
  const void *U;            // stage input: planes [nv][ncell] of the line's arithmetic
                            // (FP64, or the FP32 hi parts of the mixed form)
  void *Um, *Up;            // out: U^-_{i+1/2}, U^+_{i-1/2} of every cell, same layout and type
  void *scr;                // scratch, char_scratch_values() values of the same type
  long long ncell;          // cells per variable plane
  long long nlines;
  long long cell_stride, line_stride;
  int n;                    // cells per line
  int vn, vt;               // grid index of the normal / tangential momentum (vt < 0 in 1-D)
  int bclo, bchi;
  double gamma, eps_weno;
};

// values of one row of the scratch: the multiplier block Y (nv x nv) and
// the right-hand-side columns g (nv x (1 + nv) on periodic lines)
inline long long char_row_values(int nv, bool periodic) {
  return (long long)nv * nv + (long long)nv * (periodic ? nv + 1 : 1);
}

// scratch for lines of n cells: both sides, n rows each plus one block per
// line-side for the Woodbury coupling matrix
inline long long char_scratch_values(int nv, bool periodic, long long n, long long nlines) {
  return 2 * (n * char_row_values(nv, periodic) + (long long)nv * nv) * nlines;
}

// one launch per precision, each in its own translation unit (the FP32 one
// is compiled with the mixed form's fast division and square root)
cudaError_t launch_char_recon_f64(const CharArgs &a, int nv, bool periodic, cudaStream_t st);
cudaError_t launch_char_recon_f32(const CharArgs &a, int nv, bool periodic, cudaStream_t st);

}  // namespace ppk
