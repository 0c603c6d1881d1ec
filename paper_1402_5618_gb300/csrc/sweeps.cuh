// sweeps.cuh -- launch helpers shared by the host library and the
// per-precision translation units that instantiate the line kernel.
#pragma once

#include <cuda_runtime.h>

#include "line_sweep.cuh"

namespace ppk {

constexpr int SEG_CELLS = SEGC;   // cells per CTA of a line's cluster

struct LaunchCfg {
  int precision;   // 0 fp64, 1 mixed (fp32 line arithmetic)
  int nv;          // 3 or 4
  bool periodic;
  int mode;        // MODE_*
  bool attrs_only; // set the kernel's attributes, launch nothing
  int m;           // rows per thread chunk: 8 or 16 (picked by the autotuner)
};

// Launch one sweep over nlines lines with R CTAs per line (cluster of R);
// one entry per (precision, chunk length), each in its own translation unit.
cudaError_t launch_sweep_f64_m8(const LaunchCfg &c, const SweepArgs &a, long long nlines,
                                cudaStream_t st);
cudaError_t launch_sweep_f64_m16(const LaunchCfg &c, const SweepArgs &a, long long nlines,
                                 cudaStream_t st);
cudaError_t launch_sweep_f32_m8(const LaunchCfg &c, const SweepArgs &a, long long nlines,
                                cudaStream_t st);
cudaError_t launch_sweep_f32_m16(const LaunchCfg &c, const SweepArgs &a, long long nlines,
                                 cudaStream_t st);

// Launches with face values from another kernel (a.Fm_pre) use the M = 8
// thread layout: their kernels contain no elimination for M to tune.
inline cudaError_t launch_sweep(const LaunchCfg &c, const SweepArgs &a, long long nlines,
                                cudaStream_t st) {
  const bool m16 = c.m == 16 && !a.Fm_pre;
  if (c.precision == 0) return m16 ? launch_sweep_f64_m16(c, a, nlines, st)
                                   : launch_sweep_f64_m8(c, a, nlines, st);
  return m16 ? launch_sweep_f32_m16(c, a, nlines, st) : launch_sweep_f32_m8(c, a, nlines, st);
}

template <typename real, int NV, int M, bool PER, int MODE, bool PRE>
cudaError_t launch_m(const SweepArgs &a, long long nlines, cudaStream_t st, bool attrs_only) {
  using S = Smem<real, NV, M>;
  auto kern = line_sweep<real, NV, M, PER, MODE, PRE>;
  if (attrs_only) {   // called at handle creation, outside any stream capture
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)S::bytes);
    if (e != cudaSuccess) return e;
    // the largest shared-memory carveout, so that the resident-CTA count the
    // kernel is compiled for is not cut by the L1 split
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout,
                             (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return e;
    return cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)(nlines * a.R), 1, 1);
  cfg.blockDim = dim3(NV * S::KC, 1, 1);
  cfg.dynamicSmemBytes = S::bytes;
  cfg.stream = st;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)a.R;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, kern, a);
}

// the reconstructing kernel, or (M = 8 only) the one taking precomputed
// face values; attrs_only sets the attributes of both
template <typename real, int NV, int M, bool PER, int MODE>
cudaError_t launch_pre(const LaunchCfg &c, const SweepArgs &a, long long nlines, cudaStream_t st) {
  if constexpr (M == 8) {
    if (c.attrs_only) {
      cudaError_t e = launch_m<real, NV, M, PER, MODE, true>(a, nlines, st, true);
      if (e != cudaSuccess) return e;
    } else if (a.Fm_pre) {
      return launch_m<real, NV, M, PER, MODE, true>(a, nlines, st, false);
    }
  }
  return launch_m<real, NV, M, PER, MODE, false>(a, nlines, st, c.attrs_only);
}

template <typename real, int M>
cudaError_t launch_dispatch(const LaunchCfg &c, const SweepArgs &a, long long nlines,
                            cudaStream_t st) {
  if (c.nv == 3) {
    if (c.mode == MODE_FINAL)
      return c.periodic ? launch_pre<real, 3, M, true, MODE_FINAL>(c, a, nlines, st)
                        : launch_pre<real, 3, M, false, MODE_FINAL>(c, a, nlines, st);
    if (c.mode == MODE_OPERATOR)
      return c.periodic ? launch_pre<real, 3, M, true, MODE_OPERATOR>(c, a, nlines, st)
                        : launch_pre<real, 3, M, false, MODE_OPERATOR>(c, a, nlines, st);
    return cudaErrorInvalidValue;
  }
  if (c.nv == 4) {
    if (c.mode == MODE_XSWEEP)
      return c.periodic ? launch_pre<real, 4, M, true, MODE_XSWEEP>(c, a, nlines, st)
                        : launch_pre<real, 4, M, false, MODE_XSWEEP>(c, a, nlines, st);
    if (c.mode == MODE_FINAL)
      return c.periodic ? launch_pre<real, 4, M, true, MODE_FINAL>(c, a, nlines, st)
                        : launch_pre<real, 4, M, false, MODE_FINAL>(c, a, nlines, st);
    if (c.mode == MODE_OPERATOR)
      return c.periodic ? launch_pre<real, 4, M, true, MODE_OPERATOR>(c, a, nlines, st)
                        : launch_pre<real, 4, M, false, MODE_OPERATOR>(c, a, nlines, st);
  }
  return cudaErrorInvalidValue;
}

}  // namespace ppk
