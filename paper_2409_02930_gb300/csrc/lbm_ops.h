// Launchers of the kernel instantiations, one table per (precision, dimension).
#pragma once

#include <cuda_runtime.h>

#include "lbm_device.cuh"

namespace lbm {

template <class R> struct InletTables;
template <class R> struct StepArgs;
struct ReactArgs;

template <class R>
struct Ops {
  // two-pass form: macro-field pass, then node update reading it
  void (*macro)(const Params<R>&, const InletTables<R>&, const StepArgs<R>&, cudaStream_t);
  void (*collide)(const Params<R>&, const InletTables<R>&, const StepArgs<R>&, cudaStream_t);
  // fused single-kernel step with tile shape `variant` in [0, n_variants); returns < 0 on failure
  int (*fused)(const Params<R>&, const InletTables<R>&, const StepArgs<R>&, int variant, cudaStream_t);
  int n_variants;
  void (*init)(const Params<R>&, const double*, const double*, const double*, const double*, double, double, R*,
               const R*, cudaStream_t);
  void (*moments)(const Params<R>&, const InletTables<R>&, const StepArgs<R>&, int, double, double*, cudaStream_t);
  // reactive two-pass form (surface source); null where not instantiated
  void (*react_macro)(const Params<R>&, const InletTables<R>&, const StepArgs<R>&, const ReactArgs&, cudaStream_t);
  void (*react_collide)(const Params<R>&, const InletTables<R>&, const StepArgs<R>&, const ReactArgs&, cudaStream_t);
};

bool get_ops_f32_2d(int M, int energy, Ops<float>* out);
bool get_ops_f64_2d(int M, int energy, Ops<double>* out);
bool get_ops_f32_3d(int M, int energy, Ops<float>* out);
bool get_ops_f64_3d(int M, int energy, Ops<double>* out);

}  // namespace lbm
