// batch_lines.cuh -- descriptors of a batch of independent problems, shared
// by the line kernels and the characteristic-wise reconstruction.
#pragma once

namespace ppk {

// one problem of a batch: its block of the concatenated state (values
// [off, off + nv*ncell), variable planes of ncell cells) and grid
struct ProbDesc {
  long long off, ncell;
  int nx, ny;
  double dx, dy;
  double idx, idy;    // 1/dx, 1/dy
  int bc[4];
};

// one line of a batched launch: problem index and line index inside it
struct LineRef {
  int prob, line;
};

}  // namespace ppk
