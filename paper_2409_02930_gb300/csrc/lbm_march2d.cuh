// Pipelined fused step for D2Q9 lattices.
//
// A block of TX threads owns TX columns (TX - 2 interior columns plus one
// halo column on each side) and marches along y over SEG rows.  Every thread
// streams the pulled populations of its own column for a row into shared
// memory with asynchronous copies (cp.async, 4 or 8 bytes each; the pull
// addresses already contain the periodic wrap and the bounce-back rule), two
// rows ahead of their use, so the HBM latency is covered by the compute of
// the rows in between and no register holds a population while it is in
// flight; the porosity (and the fixed temperature of isothermal lattices) of
// every node travels the same way, so the loop issues no plain global load.
// For each row the block first computes the gradient inputs
// (u, Pi_alpha, Y_a) of all its columns into a three-row shared ring, then
// collides the interior columns of the previous row from shared memory.
// Columns next to a reservoir face take the global-memory path (their
// missing populations are reservoir equilibria computed on the fly).
#pragma once

#include "lbm_compact.cuh"

namespace lbm {

template <int BYTES>
__device__ __forceinline__ void cp_async_ca(void* smem, const void* gmem) {
  const unsigned sa = static_cast<unsigned>(__cvta_generic_to_shared(smem));
  asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// streamed values of one column, staged in shared memory [l*Q + i][TX]
template <class R, int D>
struct SmemPull {
  const R* col;
  int stride;
  static constexpr bool kUnroll = (D == 2);
  LBM_HD int prep(int, int, int) const { return 0; }
  LBM_HD R get(int, int l, int i, int, int, int) const { return col[(l * Lat<D>::Q + i) * stride]; }
};

// PD rows are prefetched ahead; PD + 2 row buffers are in use at a time
// (the static fields of each row -- porosity, and the fixed temperature of
// isothermal lattices -- travel with its populations)
template <class R, int M, bool EN, int TX, int PD>
constexpr size_t march2d_smem_bytes() {
  return sizeof(R) * (size_t)TX *
         ((PD + 2) * ((M + 1 + (EN ? 1 : 0)) * 9 + (EN ? 1 : 2)) + 3 * (4 + (EN ? M : 0)));
}

// INLET = false compiles the kernel without the reservoir-column path (for
// lattices whose x faces are periodic or bounce-back): half the code, fewer
// instruction-cache misses.
template <class R, int M, bool EN, int TX, int SEG, int MINB, int PD, bool INLET = true>
__global__ void __launch_bounds__(TX, MINB) k_march2d(Params<R> p, InletTables<R> it, StepArgs<R> a) {
  constexpr int D = 2, Q = 9;
  constexpr int NL = M + 1 + (EN ? 1 : 0);
  constexpr int NF = 2 * D + (EN ? M : 0);
  constexpr int NBUF = PD + 2;
  constexpr int NS = EN ? 1 : 2;                     // static fields per node: phi (, Tfix)
  extern __shared__ unsigned char smem_raw[];
  R* P = reinterpret_cast<R*>(smem_raw);           // [NBUF][NL*Q][TX]
  R* ring = P + (size_t)NBUF * NL * Q * TX;         // [3][NF][TX]
  R* SF = ring + (size_t)3 * NF * TX;               // [NBUF][NS][TX]

  const int t = threadIdx.x;
  const int x0 = blockIdx.x * (TX - 2);
  const int xt = x0 - 1 + t;
  int xm = xt;                                       // column whose fields this thread computes
  if (xm < 0 || xm >= p.nx) {
    const int bc = xm < 0 ? p.bc_lo : p.bc_hi;
    xm = (bc == BC_PERIODIC) ? modp(xm, p.nx) : (xm < 0 ? 0 : p.nx - 1);   // zero-gradient ghost
  }
  const bool slow = INLET && ((xm == 0 && p.bc_lo == BC_INLET) || (xm == p.nx - 1 && p.bc_hi == BC_INLET));
  const int m0 = blockIdx.y * SEG;
  const int mend = min(m0 + SEG, p.ny);
  const bool collide_col = t >= 1 && t <= TX - 2 && xt < p.nx;
  auto buf_of = [&](int row) { return (row - (m0 - 1)) % NBUF; };
  auto slot_of = [&](int row) { return (row - (m0 - 1)) % 3; };

  auto issue = [&](int row) {
    if (!slow) {
      const int y = modp(row, p.ny);
      R* dcol = P + (size_t)buf_of(row) * NL * Q * TX + t;
      R* scol = SF + (size_t)buf_of(row) * NS * TX + t;
      cp_async_ca<sizeof(R)>(scol, a.phi + xm + p.nx * y);
      if (!EN) cp_async_ca<sizeof(R)>(scol + TX, a.Tfix + xm + p.nx * y);
#pragma unroll 1
      for (int cy = -1; cy <= 1; ++cy) {
        const int sy = wrapi(y - cy, p.ny);
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx) {
          const int i = (cx + 1) + 3 * (cy + 1);
          int sx = xm - cx, isrc = i, node;
          if (sx < 0 || sx >= p.nx) {
            const int bc = sx < 0 ? p.bc_lo : p.bc_hi;
            if (bc == BC_PERIODIC) {
              node = wrapi(sx, p.nx) + p.nx * sy;
            } else {                                  // bounce-back: own opposite population
              node = xm + p.nx * y;
              isrc = Q - 1 - i;
            }
          } else {
            node = sx + p.nx * sy;
          }
#pragma unroll
          for (int l = 0; l < NL; ++l)
            cp_async_ca<sizeof(R)>(dcol + (l * Q + i) * TX, a.src + (size_t)(l * Q + isrc) * p.N + node);
        }
      }
    }
    cp_async_commit();
  };

#pragma unroll
  for (int k = 0; k < PD; ++k) issue(m0 - 1 + k);
#pragma unroll 1
  for (int s = m0 - 1; s <= mend; ++s) {
    cp_async_wait<PD - 1>();                       // row s has landed
    // ---- gradient inputs of row s (this thread's column) -------------------
    {
      const int y = modp(s, p.ny);
      const int n = xm + p.nx * y;
      Moments<R, D, M, EN, false> mo;
      if (slow) {
        Site<R, D> st;
        st.init(p, xm, y, 0);
        Ghost<R, D> gh;
        ghost_velocity<R, D, M>(p, a.src, a.phi, xm, y, 0, gh);
        moments_rt<R, D, M, EN, false>(p, it, a.src, st, gh, mo);
      } else {
        SmemPull<R, D> pf{P + (size_t)buf_of(s) * NL * Q * TX + t, TX};
        moments_gen<R, D, M, EN, false>(pf, mo);
      }
      const R* sf = SF + (size_t)buf_of(s) * NS * TX + t;
      State<R, D, M> st;
      st.template from_moments<EN, false>(p, mo, slow ? a.phi[n] : sf[0], EN ? R(0) : (slow ? a.Tfix[n] : sf[TX]));
      R* rs = ring + (size_t)slot_of(s) * NF * TX + t;
#pragma unroll
      for (int b = 0; b < D; ++b) {
        rs[b * TX] = st.u[b];
        rs[(D + b) * TX] = st.Pi(b);
      }
      if (EN) {
#pragma unroll
        for (int k = 0; k < M; ++k) rs[(2 * D + k) * TX] = st.Y[k];
      }
    }
    if (s + PD <= mend) issue(s + PD);
    else cp_async_commit();
    __syncthreads();
    // ---- collide row s - 1 ---------------------------------------------------
    if (s - 1 >= m0 && collide_col) {
      const int y = s - 1;
      const int n = xt + p.nx * y;
      Moments<R, D, M, EN, true> mo;
      Site<R, D> site;
      site.init(p, xt, y, 0);
      Ghost<R, D> gh;
      gh.side = -1;
      if (slow) {
        ghost_velocity<R, D, M>(p, a.src, a.phi, xt, y, 0, gh);
        moments_rt<R, D, M, EN, true>(p, it, a.src, site, gh, mo);
      } else {
        SmemPull<R, D> pf{P + (size_t)buf_of(y) * NL * Q * TX + t, TX};
        moments_gen<R, D, M, EN, true>(pf, mo);
      }
      // this thread's ring column is its collide column (xm == xt here)
      const R* sf = SF + (size_t)buf_of(y) * NS * TX + t;
      State<R, D, M> st;
      st.template from_moments<EN, true>(p, mo, slow ? a.phi[n] : sf[0], EN ? R(0) : (slow ? a.Tfix[n] : sf[TX]));
      Grad<R, D, M, EN> gr;
      gr.divu = R(0);
#pragma unroll
      for (int b = 0; b < D; ++b) {
        gr.dPi[b] = R(0);
#pragma unroll
        for (int k = 0; k < M; ++k) gr.dY[k][b] = R(0);
      }
#pragma unroll
      for (int cy = -1; cy <= 1; ++cy) {
        const R* rr = ring + (size_t)slot_of(y + cy) * NF * TX + t;
#pragma unroll
        for (int cx = -1; cx <= 1; ++cx) {
          if (cx == 0 && cy == 0) continue;
          const R w = R(3) * (cx == 0 ? R(2) / R(3) : R(1) / R(6)) * (cy == 0 ? R(2) / R(3) : R(1) / R(6));
          if (cx != 0) {
            const R wc = w * R(cx);
            gr.divu += wc * rr[cx];
            gr.dPi[0] += wc * rr[D * TX + cx];
            if (EN) {
#pragma unroll
              for (int k = 0; k < M; ++k) gr.dY[k][0] += wc * rr[(2 * D + k) * TX + cx];
            }
          }
          if (cy != 0) {
            const R wc = w * R(cy);
            gr.divu += wc * rr[TX + cx];
            gr.dPi[1] += wc * rr[(D + 1) * TX + cx];
            if (EN) {
#pragma unroll
              for (int k = 0; k < M; ++k) gr.dY[k][1] += wc * rr[(2 * D + k) * TX + cx];
            }
          }
        }
      }
      if (slow) {
        GlobalPull<R, D, M, EN> pf{p, it, a.src, site, gh};
        collide_gen<R, D, M, EN>(p, pf, n, mo, st, gr, a.dst, a.status);
      } else {
        SmemPull<R, D> pf{P + (size_t)buf_of(y) * NL * Q * TX + t, TX};
        collide_gen<R, D, M, EN>(p, pf, n, mo, st, gr, a.dst, a.status);
      }
    }
    __syncthreads();
  }
  cp_async_wait<0>();
}

}  // namespace lbm
