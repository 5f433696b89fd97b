// Fused single-kernel time step.
//
// A block owns a tile of TX (x) by TY (y, 3-D only) nodes and marches along
// the slowest axis (y in 2-D, z in 3-D) over SEG planes.  For every plane it
// first recomputes, from the streamed populations, the macroscopic fields
// that the isotropic gradients need (u, Pi_alpha of Eq. 45, Y_a) on the tile
// plus a one-node halo, into a rolling shared-memory ring of three planes;
// then it collides the interior nodes of the previous plane, whose stencil
// now lies entirely in the ring.  No macro field goes through global memory,
// so the populations are read from HBM about once per step (the halo
// re-reads hit L2) and written once.
#pragma once

#include "lbm_compact.cuh"

namespace lbm {

template <int D, int M, bool EN>
struct FusedLayout {
  static constexpr int NF = 2 * D + (EN ? M : 0);
};

template <class R, int D, int M, bool EN, int TX, int TY>
constexpr size_t fused_smem_bytes() {
  return sizeof(R) * 3 * FusedLayout<D, M, EN>::NF * (TX + 2) * ((D == 3) ? TY + 2 : 1);
}

LBM_HD int modp(int v, int n) {
  int r = v % n;
  return r < 0 ? r + n : r;
}

template <class R, int D, int M, bool EN, int TX, int TY, int SEG>
__global__ void __launch_bounds__(TX * TY) k_fused(Params<R> p, InletTables<R> it, StepArgs<R> a) {
  constexpr int NT = TX * TY;
  constexpr int PX = TX + 2;
  constexpr int PY = (D == 3) ? TY + 2 : 1;
  constexpr int PN = PX * PY;
  constexpr int NF = FusedLayout<D, M, EN>::NF;
  extern __shared__ unsigned char smem_raw[];
  R* ring = reinterpret_cast<R*>(smem_raw);           // [3][NF][PN]

  const int x0 = blockIdx.x * TX;
  const int y0 = (D == 3) ? blockIdx.y * TY : 0;
  const int m0 = ((D == 3) ? blockIdx.z : blockIdx.y) * SEG;
  const int mlen = (D == 3) ? p.nz : p.ny;
  const int mend = min(m0 + SEG, mlen);
  const int tid = threadIdx.x;

  // macro fields of one extended plane (march coordinate m) into a ring slot
  auto compute_plane = [&](int m, int slot) {
    const int mw = modp(m, mlen);
    R* dstp = ring + (size_t)slot * NF * PN;
    for (int e = tid; e < PN; e += NT) {
      const int ex = e % PX, ey = e / PX;
      int x = x0 - 1 + ex;
      if (x < 0 || x >= p.nx) {
        const int bc = x < 0 ? p.bc_lo : p.bc_hi;
        x = (bc == BC_PERIODIC) ? modp(x, p.nx) : (x < 0 ? 0 : p.nx - 1);   // zero-gradient ghost
      }
      int y, z;
      if (D == 3) {
        y = modp(y0 - 1 + ey, p.ny);
        z = mw;
      } else {
        y = mw;
        z = 0;
      }
      Site<R, D> st;
      st.init(p, x, y, z);
      Ghost<R, D> gh;
      gh.side = -1;
      if (st.has_ghost()) ghost_velocity<R, D, M>(p, a.src, a.phi, x, y, z, gh);
      Moments<R, D, M, EN, false> mo;
      moments_rt<R, D, M, EN, false>(p, it, a.src, st, gh, mo);
      State<R, D, M> s;
      s.template from_moments<EN, false>(p, mo, a.phi[st.n], EN ? R(0) : a.Tfix[st.n]);
#pragma unroll
      for (int b = 0; b < D; ++b) {
        dstp[b * PN + e] = s.u[b];
        dstp[(D + b) * PN + e] = s.Pi(b);
      }
      if (EN) {
#pragma unroll
        for (int k = 0; k < M; ++k) dstp[(2 * D + k) * PN + e] = s.Y[k];
      }
    }
  };
  auto slot_of = [](int r) { return (r + 1) % 3; };    // r = m - m0 in [-1, SEG]

  const int tx = tid % TX, ty = tid / TX;
  const int xi = x0 + tx;
  const int yi = (D == 3) ? y0 + ty : 0;
  const bool active = xi < p.nx && (D == 2 || yi < p.ny);

  compute_plane(m0 - 1, slot_of(-1));
  compute_plane(m0, slot_of(0));
  for (int r = 0; r < mend - m0; ++r) {
    compute_plane(m0 + r + 1, slot_of(r + 1));
    __syncthreads();
    if (active) {
      const int m = m0 + r;
      const int x = xi, y = (D == 3) ? yi : m, z = (D == 3) ? m : 0;
      Site<R, D> st;
      st.init(p, x, y, z);
      Ghost<R, D> gh;
      gh.side = -1;
      if (st.has_ghost()) ghost_velocity<R, D, M>(p, a.src, a.phi, x, y, z, gh);
      Moments<R, D, M, EN, true> mo;
      moments_rt<R, D, M, EN, true>(p, it, a.src, st, gh, mo);
      State<R, D, M> s;
      s.template from_moments<EN, true>(p, mo, a.phi[st.n], EN ? R(0) : a.Tfix[st.n]);
      // gradient inputs from the ring (isotropic stencil, weights 3 w_i)
      Grad<R, D, M, EN> gr;
      gr.divu = R(0);
#pragma unroll
      for (int b = 0; b < D; ++b) {
        gr.dPi[b] = R(0);
#pragma unroll
        for (int k = 0; k < M; ++k) gr.dY[k][b] = R(0);
      }
      for_each_dir<D>([&](int i, int cx, int cy, int cz) {
        const int c2 = cx * cx + cy * cy + cz * cz;
        if (c2 == 0) return;
        const R w = R(3) * (cx == 0 ? R(2) / R(3) : R(1) / R(6)) * (cy == 0 ? R(2) / R(3) : R(1) / R(6)) *
                    ((D == 3) ? (cz == 0 ? R(2) / R(3) : R(1) / R(6)) : R(1));
        const int dm = (D == 3) ? cz : cy;                 // march-axis offset
        const int e = (D == 3) ? (ty + 1 + cy) * PX + (tx + 1 + cx) : (tx + 1 + cx);
        const R* src_pl = ring + (size_t)slot_of(r + dm) * NF * PN;
        const int cc[3] = {cx, cy, cz};
#pragma unroll
        for (int b = 0; b < D; ++b) {
          if (cc[b] == 0) continue;
          const R wc = w * R(cc[b]);
          gr.divu += wc * src_pl[b * PN + e];
          gr.dPi[b] += wc * src_pl[(D + b) * PN + e];
          if (EN) {
#pragma unroll
            for (int k = 0; k < M; ++k) gr.dY[k][b] += wc * src_pl[(2 * D + k) * PN + e];
          }
        }
      });
      collide_rt<R, D, M, EN>(p, it, a.src, st, gh, mo, s, gr, a.dst, a.status);
    }
    __syncthreads();
  }
}

}  // namespace lbm
