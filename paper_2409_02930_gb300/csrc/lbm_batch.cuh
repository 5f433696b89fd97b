// Batched form: many independent 2-D lattices (capillaries or slabs of
// uneven size and pressure, each with its own lattice scaling) advanced by
// persistent kernels over one work list of node tiles.
//
// Every case keeps the single-lattice layout ([L][Q][N_c] populations,
// [2D+M][N_c] macro fields) at its own offset inside shared buffers, so the
// per-node code of the two-pass step (lbm_kernels.cuh) runs unchanged with
// the case's own parameters (read through the L1 cache from the case table).
// A block takes a contiguous range of the tile list, which keeps most of its
// tiles inside one case.
#pragma once

#include "lbm_kernels.cuh"
#include "lbm_staged.cuh"

namespace lbm {

template <class R>
struct CaseDev {
  Params<R> p;
  InletTables<R> it;
  long long pop_off;    // element offset of the case's populations
  long long node_off;   // offset of its per-node fields (porosity, temperature)
  long long mac_off;    // offset of its macro-field block
};

template <class R>
struct BatchArgs {
  const CaseDev<R>* cases;
  const int2* tiles;    // (case, first node of the tile)
  int ntiles;
  const R* src;
  R* dst;
  const R* phi;
  const R* Tfix;
  R* mac;
  int* status;
};

// One pass of the two-pass step over every tile: COLLIDE = false computes the
// macro fields, COLLIDE = true the node update.  Tiles are TB nodes long.
template <class R, int D, int M, bool EN, int TB, bool COLLIDE>
__global__ void __launch_bounds__(TB) k_batch(BatchArgs<R> b) {
  const int t0 = (int)((long long)blockIdx.x * b.ntiles / gridDim.x);
  const int t1 = (int)((long long)(blockIdx.x + 1) * b.ntiles / gridDim.x);
  for (int t = t0; t < t1; ++t) {
    const int2 tl = b.tiles[t];
    const CaseDev<R>& cs = b.cases[tl.x];
    const int n = tl.y + (int)threadIdx.x;
    if (n >= cs.p.N) continue;
    StepArgs<R> a{b.src + cs.pop_off, b.dst + cs.pop_off, b.phi + cs.node_off, b.Tfix + cs.node_off,
                  b.mac + cs.mac_off, b.status};
    if (COLLIDE) collide_node<R, D, M, EN>(cs.p, cs.it, a, n);
    else macro_node<R, D, M, EN>(cs.p, cs.it, a, n);
  }
}

// The same passes with every node's pulled populations staged in shared
// memory (TB x L*Q values per block; a thread reuses its column for each of
// its tiles).
template <class R, int D, int M, bool EN, int TB, bool COLLIDE>
__global__ void __launch_bounds__(TB) k_batch_staged(BatchArgs<R> b) {
  extern __shared__ unsigned char smem_raw[];
  R* col = reinterpret_cast<R*>(smem_raw) + threadIdx.x;
  const int t0 = (int)((long long)blockIdx.x * b.ntiles / gridDim.x);
  const int t1 = (int)((long long)(blockIdx.x + 1) * b.ntiles / gridDim.x);
  for (int t = t0; t < t1; ++t) {
    const int2 tl = b.tiles[t];
    const CaseDev<R>& cs = b.cases[tl.x];
    const int n = tl.y + (int)threadIdx.x;
    if (n >= cs.p.N) continue;
    StepArgs<R> a{b.src + cs.pop_off, b.dst + cs.pop_off, b.phi + cs.node_off, b.Tfix + cs.node_off,
                  b.mac + cs.mac_off, b.status};
    if (COLLIDE) collide_staged_node<R, D, M, EN>(cs.p, cs.it, a, n, col, TB);
    else macro_staged_node<R, D, M, EN>(cs.p, cs.it, a, n, col, TB);
  }
}

// Launch table of the batched form for one (precision, M, energy).
template <class R>
struct BatchOps {
  // tile length (= block size) of variant v
  int (*tile)(int v);
  // resident blocks per SM of the kernels of variant v (occupancy query)
  int (*occupancy)(int v);
  // one pass of a time step (collide = 0: macro fields, 1: node update) with
  // variant v on grid blocks
  void (*pass)(const BatchArgs<R>&, int v, int grid, int collide, cudaStream_t);
  int n_variants;
};

bool get_batch_ops_f32(int M, int energy, BatchOps<float>* out);
bool get_batch_ops_f64(int M, int energy, BatchOps<double>* out);

}  // namespace lbm
