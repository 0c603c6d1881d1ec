// char_recon.cuh -- the characteristic-wise compact-WENO reconstruction of
// one sweep direction (Sec. 2.3, steps 1-4, eqs. (cha-1), (1DEuler-FVC)).
//
// For every line and each side (minus: U^-_{i+1/2}, plus: U^+_{i-1/2}) the
// block tridiagonal system of the line is assembled and solved in two
// kernels.  The first runs over every row of every line in parallel: the
// Roe average of the two cells adjacent to the row's face, its left
// eigenvectors l^(k) (eq. (leigenv); the 4 x 4 system with the shear field in
// 2-D), the characteristic variables l^(k) ubar of the five-cell stencil, and
// per field the WENO-Z weights and scalar row coefficients (a, b, c, r).  The
// second walks each line in the stable elimination order (minus left to
// right, plus right to left), one thread per (line, side), forming the block
// row diag(a, b, c) L and one block Thomas step per position; only that
// recurrence is serial.  The multipliers go to a scratch buffer laid out
// [row][entry][line] so that the threads of a warp (consecutive lines) access
// it together.  Periodic lines carry the Woodbury columns of the cyclic
// correction through the same pass.  Bounded lines close the first and last
// unknown with the explicit WENO5-Z value of each characteristic variable at
// that face.
//
// The output planes hold U^- and U^+ of every cell in the state's layout and
// grid variable order; the line kernel limits them, evaluates the face
// fluxes and forms the stage update.
#pragma once

#include <cuda_runtime.h>

#include "batch_lines.cuh"

namespace ppk {

struct CharArgs {
  const void *U;            // stage input: planes [nv][ncell] of the line's arithmetic
                            // (FP64, or the FP32 hi parts of the mixed form)
  void *Um, *Up;            // out: U^-_{i+1/2}, U^+_{i-1/2} of every cell, same layout and type
  void *scr;                // block Thomas scratch, char_scratch_values() values of the same type
  void *rows;               // row coefficients, char_rows_values() values of the same type
  long long ncell;          // cells per variable plane
  long long nlines;
  long long cell_stride, line_stride;
  int n;                    // cells per line; batched: the longest line (position stride of rows, scr)
  int vn, vt;               // grid index of the normal / tangential momentum (vt < 0 in 1-D)
  int bclo, bchi;
  double gamma, eps_weno;
  // batched launch (nullptr: one problem): the group's line table and the
  // problem descriptors; each line takes its length, boundaries and slice
  // of U, Um, Up from its problem
  const LineRef *lines;
  const ProbDesc *probs;
  int xdir;                 // batched: 1 x lines, 0 y lines (columns), 2 rows of the transposed planes
  int layout;               // FP32 block solve: 0 one thread per walk, 1 four lanes per walk,
                            // < 0 by the number of walks (four lanes below 2048 lines)
};

// values of one row of the scratch: the multiplier block Y (nv x nv) and
// the right-hand-side columns g (nv x (1 + nv) on periodic lines)
inline long long char_row_values(int nv, bool periodic) {
  return (long long)nv * nv + (long long)nv * (periodic ? nv + 1 : 1);
}

// scratch for lines of (at most) n cells: both sides, n rows each plus one
// block per line-side for the Woodbury coupling matrix
inline long long char_scratch_values(int nv, bool periodic, long long n, long long nlines) {
  return 2 * (n * char_row_values(nv, periodic) + (long long)nv * nv) * nlines;
}

// row data of every row of both sides: the four Roe scalars the
// eigenvectors depend on and (a, b, c, r) of every field
inline long long char_rows_values(int nv, long long n, long long nlines) {
  return 2 * (4 * (long long)nv + 4) * n * nlines;
}

// one entry per precision, each in its own translation unit (the FP32 one
// is compiled with the mixed form's fast division and square root); part 0
// launches the parallel rows kernel, part 1 the serial block solve
cudaError_t launch_char_recon_f64(const CharArgs &a, int nv, bool periodic, int part, cudaStream_t st);
cudaError_t launch_char_recon_f32(const CharArgs &a, int nv, bool periodic, int part, cudaStream_t st);

}  // namespace ppk
