// Node update of the two-pass form with the node's streamed populations
// staged in shared memory.  Every thread issues the asynchronous copies of
// all its pulled populations (L*Q of them; the pull addresses already hold
// the periodic wrap and the bounce-back rule; reservoir ghosts are computed
// and stored directly), waits once, and collides from shared memory.  With
// 216 populations per node (D3Q27, six species, energy) the copies of a node
// are all in flight together instead of one dependent load per direction.
#pragma once

#include "lbm_compact.cuh"
#include "lbm_march2d.cuh"
#include "lbm_surface.cuh"

namespace lbm {

// populations per node
template <class R, int D, int M, bool EN>
constexpr int n_pops() {
  return (M + 1 + (EN ? 1 : 0)) * Lat<D>::Q;
}

// Stages the pulled populations of node (x, y, z) into col[(l*Q + i) * stride].
template <class R, int D, int M, bool EN>
__device__ __forceinline__ void stage_node(const Params<R>& p, const InletTables<R>& it, const R* __restrict__ src,
                                           const Site<R, D>& st, const Ghost<R, D>& gh, R* col, int stride) {
  constexpr int Q = Lat<D>::Q, L = M + 1 + (EN ? 1 : 0);
  const size_t N = p.N;
  for_each_dir<D>([&](int i, int cx, int cy, int cz) {
    const int h = st.source(cx, cy, cz);
    if (h == SRC_GHOST) {
#pragma unroll
      for (int l = 0; l < L; ++l)
        col[(l * Q + i) * stride] = pull_rt<R, D, M, EN>(p, it, src, gh, st.n, h, l, i, cx, cy, cz);
    } else {
      const int node = h >= 0 ? h : -1 - h;          // bounce-back: the node's own opposite population
      const int isrc = h >= 0 ? i : Q - 1 - i;
#pragma unroll
      for (int l = 0; l < L; ++l)
        cp_async_ca<sizeof(R)>(col + (l * Q + i) * stride, src + (size_t)(l * Q + isrc) * N + node);
    }
  });
  cp_async_commit();
  cp_async_wait<0>();
}

// Moments, state and gradient inputs of a staged node.
template <class R, int D, int M, bool EN>
__device__ __forceinline__ void staged_state(const Params<R>& p, const StepArgs<R>& a, const SmemPull<R, D>& pf,
                                             int n, int x, int y, int z, Moments<R, D, M, EN, true>& mo,
                                             State<R, D, M>& s, Grad<R, D, M, EN>& gr) {
  moments_gen<R, D, M, EN, true>(pf, mo);
  s.template from_moments<EN, true>(p, mo, a.phi[n], EN ? R(0) : a.Tfix[n]);
  const R* __restrict__ mac = a.mac;
  const int N = p.N;
  gr.compute(p, x, y, z, [&](int k, int nb) { return mac[(size_t)k * N + nb]; });
}

// Macro fields of node n (u, Pi_alpha, Y_a for the neighbours' gradients)
// from its populations staged in col[(l*Q + i) * stride].
template <class R, int D, int M, bool EN>
__device__ __forceinline__ void macro_staged_node(const Params<R>& p, const InletTables<R>& it, const StepArgs<R>& a,
                                                  int n, R* col, int stride) {
  int x, y, z;
  node_xyz<R, D>(p, n, x, y, z);
  Site<R, D> st;
  st.init(p, x, y, z);
  Ghost<R, D> gh;
  gh.side = -1;
  if (st.has_ghost()) ghost_velocity<R, D, M>(p, a.src, a.phi, x, y, z, gh);
  stage_node<R, D, M, EN>(p, it, a.src, st, gh, col, stride);
  SmemPull<R, D> pf{col, stride};
  Moments<R, D, M, EN, false> mo;
  moments_gen<R, D, M, EN, false>(pf, mo);
  State<R, D, M> s;
  s.template from_moments<EN, false>(p, mo, a.phi[n], EN ? R(0) : a.Tfix[n]);
  const size_t N = p.N;
#pragma unroll
  for (int b = 0; b < D; ++b) {
    a.mac[(size_t)b * N + n] = s.u[b];
    a.mac[(size_t)(D + b) * N + n] = s.Pi(b);
  }
  if (EN) {
#pragma unroll
    for (int k = 0; k < M; ++k) a.mac[(size_t)(2 * D + k) * N + n] = s.Y[k];
  }
}

// Node update of node n from its staged populations.
template <class R, int D, int M, bool EN>
__device__ __forceinline__ void collide_staged_node(const Params<R>& p, const InletTables<R>& it,
                                                    const StepArgs<R>& a, int n, R* col, int stride) {
  int x, y, z;
  node_xyz<R, D>(p, n, x, y, z);
  Site<R, D> st;
  st.init(p, x, y, z);
  Ghost<R, D> gh;
  gh.side = -1;
  if (st.has_ghost()) ghost_velocity<R, D, M>(p, a.src, a.phi, x, y, z, gh);
  stage_node<R, D, M, EN>(p, it, a.src, st, gh, col, stride);
  SmemPull<R, D> pf{col, stride};
  Moments<R, D, M, EN, true> mo;
  State<R, D, M> s;
  Grad<R, D, M, EN> gr;
  staged_state<R, D, M, EN>(p, a, pf, n, x, y, z, mo, s, gr);
  collide_gen<R, D, M, EN>(p, pf, n, mo, s, gr, a.dst, a.status);
}

// Gradient inputs of every node (divu, dPi_b and, with energy, dY_a,b) in a
// pass of their own, written after the macro fields at
// mac + (2D + M) N as [1 + D + M D][N]: the node update then reads NG
// coalesced values instead of gathering the macro fields of its 26 (8)
// neighbours.  Same stencil code and order as the gathering form.
template <int D, int M, bool EN>
constexpr int n_grad_fields() {
  return 1 + D + (EN ? M * D : 0);
}

template <class R, int D, int M, bool EN>
__global__ void __launch_bounds__(256) k_grad(Params<R> p, StepArgs<R> a) {
  const int n = blockIdx.x * blockDim.x + threadIdx.x;
  if (n >= p.N) return;
  int x, y, z;
  node_xyz<R, D>(p, n, x, y, z);
  const R* __restrict__ mac = a.mac;
  const size_t N = p.N;
  Grad<R, D, M, EN> gr;
  gr.compute(p, x, y, z, [&](int k, int nb) { return mac[(size_t)k * N + nb]; });
  R* g = a.mac + (size_t)(2 * D + M) * N;
  g[n] = gr.divu;
#pragma unroll
  for (int b = 0; b < D; ++b) g[(size_t)(1 + b) * N + n] = gr.dPi[b];
  if (EN) {
#pragma unroll
    for (int k = 0; k < M; ++k)
#pragma unroll
      for (int b = 0; b < D; ++b) g[(size_t)(1 + D + k * D + b) * N + n] = gr.dY[k][b];
  }
}

// Node update of node n from its staged populations and the gradient inputs
// of the gradient pass.
template <class R, int D, int M, bool EN>
__device__ __forceinline__ void collide_staged_node_g(const Params<R>& p, const InletTables<R>& it,
                                                      const StepArgs<R>& a, int n, R* col, int stride) {
  int x, y, z;
  node_xyz<R, D>(p, n, x, y, z);
  Site<R, D> st;
  st.init(p, x, y, z);
  Ghost<R, D> gh;
  gh.side = -1;
  if (st.has_ghost()) ghost_velocity<R, D, M>(p, a.src, a.phi, x, y, z, gh);
  stage_node<R, D, M, EN>(p, it, a.src, st, gh, col, stride);
  SmemPull<R, D> pf{col, stride};
  Moments<R, D, M, EN, true> mo;
  moments_gen<R, D, M, EN, true>(pf, mo);
  State<R, D, M> s;
  s.template from_moments<EN, true>(p, mo, a.phi[n], EN ? R(0) : a.Tfix[n]);
  const size_t N = p.N;
  const R* __restrict__ g = a.mac + (size_t)(2 * D + M) * N;
  Grad<R, D, M, EN> gr;
  gr.divu = g[n];
#pragma unroll
  for (int b = 0; b < D; ++b) {
    gr.dPi[b] = g[(size_t)(1 + b) * N + n];
#pragma unroll
    for (int k = 0; k < M; ++k) gr.dY[k][b] = EN ? g[(size_t)(1 + D + k * D + b) * N + n] : R(0);
  }
  collide_gen<R, D, M, EN>(p, pf, n, mo, s, gr, a.dst, a.status);
}

template <class R, int D, int M, bool EN, int TB>
__global__ void __launch_bounds__(TB) k_collide_staged_g(Params<R> p, InletTables<R> it, StepArgs<R> a) {
  extern __shared__ unsigned char smem_raw[];
  const int n = blockIdx.x * TB + threadIdx.x;
  if (n >= p.N) return;
  collide_staged_node_g<R, D, M, EN>(p, it, a, n, reinterpret_cast<R*>(smem_raw) + threadIdx.x, TB);
}

// Macro-field pass from staged populations.
template <class R, int D, int M, bool EN, int TB>
__global__ void __launch_bounds__(TB) k_macro_staged(Params<R> p, InletTables<R> it, StepArgs<R> a) {
  extern __shared__ unsigned char smem_raw[];
  const int n = blockIdx.x * TB + threadIdx.x;
  if (n >= p.N) return;
  macro_staged_node<R, D, M, EN>(p, it, a, n, reinterpret_cast<R*>(smem_raw) + threadIdx.x, TB);
}

template <class R, int D, int M, bool EN, int TB>
__global__ void __launch_bounds__(TB) k_collide_staged(Params<R> p, InletTables<R> it, StepArgs<R> a) {
  extern __shared__ unsigned char smem_raw[];
  const int n = blockIdx.x * TB + threadIdx.x;
  if (n >= p.N) return;
  collide_staged_node<R, D, M, EN>(p, it, a, n, reinterpret_cast<R*>(smem_raw) + threadIdx.x, TB);
}

// Reactive node update (surface sources of the first pass) from staged populations.
template <class R, int D, int M, bool EN, int TB>
__global__ void __launch_bounds__(TB) k_collide_react_staged(Params<R> p, InletTables<R> it, StepArgs<R> a,
                                                             ReactArgs ra) {
  extern __shared__ unsigned char smem_raw[];
  R* col = reinterpret_cast<R*>(smem_raw) + threadIdx.x;
  const int n = blockIdx.x * TB + threadIdx.x;
  if (n >= p.N) return;
  int x, y, z;
  node_xyz<R, D>(p, n, x, y, z);
  Site<R, D> st;
  st.init(p, x, y, z);
  Ghost<R, D> gh;
  gh.side = -1;
  if (st.has_ghost()) ghost_velocity<R, D, M>(p, a.src, a.phi, x, y, z, gh);
  stage_node<R, D, M, EN>(p, it, a.src, st, gh, col, TB);
  SmemPull<R, D> pf{col, TB};
  Moments<R, D, M, EN, true> mo;
  State<R, D, M> s;
  Grad<R, D, M, EN> gr;
  staged_state<R, D, M, EN>(p, a, pf, n, x, y, z, mo, s, gr);
  const int N = p.N;
  NodeSource<R> srcv;
  for (int k = 0; k < M; ++k) srcv.rhodot[k] = (R)ra.src[(size_t)k * N + n];
  srcv.dU = (R)ra.src[(size_t)M * N + n];
  collide_gen<R, D, M, EN, SmemPull<R, D>, true>(p, pf, n, mo, s, gr, a.dst, a.status, &srcv);
}

}  // namespace lbm
