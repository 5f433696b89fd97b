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
#include "lbm_tma.cuh"

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

// Row-box layout of the TMA form: for each row buffer, one chunk per
// direction i holding the source row y - c_iy of every lattice over W columns
// starting at xs (a 16-byte aligned column at or left of x0 - 2), then the
// static-field rows.  Each chunk starts on a 128-byte boundary, as the bulk
// tensor copies want.  Thread t reads direction i of lattice l at
// [i][l][t + c0 - c_ix] with c0 = x0 - 1 - xs.
template <class R, int M, bool EN, int TX, int PD>
struct RowBoxLayout {
  static constexpr int NL = M + 1 + (EN ? 1 : 0);
  static constexpr int NS = EN ? 1 : 2;
  static constexpr int AU = 16 / (int)sizeof(R);          // elements per 16 bytes
  static constexpr int A128 = 128 / (int)sizeof(R);       // elements per 128 bytes
  static constexpr int W = ((TX + 1 + AU + AU - 1) / AU) * AU;
  static constexpr int CH = ((NL * W + A128 - 1) / A128) * A128;
  static constexpr int SCH = ((W + A128 - 1) / A128) * A128;
  static constexpr int BUFE = 9 * CH + NS * SCH;          // elements per row buffer
  static constexpr int NBUF = PD + 2;
  static constexpr int NF = 4 + (EN ? M : 0);
  static constexpr uint32_t kRowBytes = (uint32_t)sizeof(R) * W * (9 * NL + NS);   // bytes landing per row
  static constexpr size_t bytes() {
    return 128 + sizeof(R) * ((size_t)NBUF * BUFE + 3 * (size_t)NF * TX) + 8 * (size_t)(NBUF + 1);
  }
};

// streamed values of one column in the row-box layout
template <class R, int CH, int LW>
struct RowPull {
  const R* col;                      // chunk base + t + c0
  static constexpr bool kUnroll = true;
  LBM_HD int prep(int, int, int) const { return 0; }
  LBM_HD R get(int, int l, int i, int cx, int, int) const { return col[i * CH + l * LW - cx]; }
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
//
// TMA = true stages each row with bulk tensor copies issued by one thread
// (nine row boxes of every lattice, one per direction, plus the static-field
// rows) completing on an mbarrier per row buffer, instead of one cp.async per
// population and thread.  Blocks whose columns reach past an x face (the
// periodic wrap and the bounce-back rule live in the per-thread addresses)
// stage with per-thread cp.async into the same row-box layout.  The waits are
// bounded: a wait that gives up sets the timeout status bit, ends the march
// and drains the copies still in flight (again bounded) before returning.
template <class R, int M, bool EN, int TX, int SEG, int MINB, int PD, bool INLET = true, bool TMA = false>
__global__ void __launch_bounds__(TX, MINB)
    k_march2d(Params<R> p, InletTables<R> it, StepArgs<R> a, const __grid_constant__ TmaMaps tm) {
  constexpr int D = 2, Q = 9;
  constexpr int NL = M + 1 + (EN ? 1 : 0);
  constexpr int NF = 2 * D + (EN ? M : 0);
  constexpr int NBUF = PD + 2;
  constexpr int NS = EN ? 1 : 2;                     // static fields per node: phi (, Tfix)
  using LB = RowBoxLayout<R, M, EN, TX, PD>;
  extern __shared__ unsigned char smem_raw[];
  unsigned char* sbase = smem_raw;
  if constexpr (TMA)
    sbase = smem_raw + ((128 - (smem_u32(smem_raw) & 127)) & 127);
  R* P = reinterpret_cast<R*>(sbase);               // [NBUF][NL*Q][TX], or [NBUF][BUFE] (TMA)
  constexpr size_t PE = TMA ? (size_t)LB::BUFE : (size_t)NL * Q * TX;
  R* ring = P + (size_t)NBUF * PE;                  // [3][NF][TX]
  R* SF = ring + (size_t)3 * NF * TX;               // [NBUF][NS][TX] (cp.async layout)
  uint64_t* bar = reinterpret_cast<uint64_t*>(
      (reinterpret_cast<uintptr_t>(ring + (size_t)3 * NF * TX) + 7) & ~(uintptr_t)7);   // [NBUF] (TMA)

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
  // TMA form: first staged column, this thread's offset into a row box, and
  // whether the block stages with bulk copies (all its source columns inside)
  const int xs = TMA ? ((x0 - 2 >= 0) ? (x0 - 2) / LB::AU * LB::AU : -LB::AU) : 0;
  const int c0 = x0 - 1 - xs;
  const bool bulk = TMA && x0 - 2 >= 0 && x0 + TX - 1 <= p.nx - 1;
  // column base of this thread in row buffer b
  auto col_of = [&](int b) -> R* {
    return TMA ? P + (size_t)b * PE + t + c0 : P + (size_t)b * PE + t;
  };
  auto static_of = [&](int b) -> const R* {
    return TMA ? P + (size_t)b * PE + 9 * LB::CH + t + c0 : SF + (size_t)b * NS * TX + t;
  };
  constexpr int SSTR = TMA ? LB::SCH : TX;           // distance of Tfix from phi

  if constexpr (TMA) {
    if (bulk && t == 0) {
      for (int b = 0; b < NBUF; ++b) mbar_init(bar + b, 1);
      mbar_fence_init();
    }
    __syncthreads();
  }

  auto issue = [&](int row) {
    const int y = modp(row, p.ny);
    if (TMA && bulk) {
      if (t == 0) {
        const int b = buf_of(row);
        R* dst = P + (size_t)b * PE;
        fence_proxy_async_smem();
        mbar_arrive_expect_tx(bar + b, LB::kRowBytes);
#pragma unroll 1
        for (int i = 0; i < Q; ++i) {
          const int cy = i / 3 - 1;
          tma_load_4d(dst + i * LB::CH, &tm.pop, xs, wrapi(y - cy, p.ny), i, 0, bar + b);
        }
        tma_load_2d(dst + 9 * LB::CH, &tm.phi, xs, y, bar + b);
        if (!EN) tma_load_2d(dst + 9 * LB::CH + LB::SCH, &tm.T, xs, y, bar + b);
      }
      return;
    }
    if (!slow) {
      R* dcol = col_of(buf_of(row));
      R* scol = const_cast<R*>(static_of(buf_of(row)));
      cp_async_ca<sizeof(R)>(scol, a.phi + xm + p.nx * y);
      if (!EN) cp_async_ca<sizeof(R)>(scol + SSTR, a.Tfix + xm + p.nx * y);
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
          for (int l = 0; l < NL; ++l) {
            R* d = TMA ? dcol + i * LB::CH + l * LB::W - cx : dcol + (l * Q + i) * TX;
            cp_async_ca<sizeof(R)>(d, a.src + (size_t)(l * Q + isrc) * p.N + node);
          }
        }
      }
    }
    cp_async_commit();
  };
  // waits until row `row` has landed in its buffer; false if a bounded wait gave up
  auto landed = [&](int row) -> bool {
    if (TMA && bulk) return mbar_wait(bar + buf_of(row), (uint32_t)(((row - (m0 - 1)) / NBUF) & 1), p.wait_limit);
    cp_async_wait<PD - 1>();
    return true;
  };

#pragma unroll
  for (int k = 0; k < PD; ++k) issue(m0 - 1 + k);
  int last_issued = m0 - 1 + PD - 1;
  int aborted_at = mend + 1;
  // Without reservoir columns the state a thread computes for its column in
  // the ring phase of row s (from the same zeroth and first moments, in the
  // same order) is the state the collision of row s needs one iteration
  // later: it is kept in registers instead of being formed again.
  constexpr bool KEEP = TMA && !INLET;
  State<R, D, M> st_prev, st_new;
#pragma unroll 1
  for (int s = m0 - 1; s <= mend; ++s) {
    const bool ok = landed(s);                       // row s has landed
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
      } else if constexpr (TMA) {
        RowPull<R, LB::CH, LB::W> pf{col_of(buf_of(s))};
        moments_gen<R, D, M, EN, false>(pf, mo);
      } else {
        SmemPull<R, D> pf{col_of(buf_of(s)), TX};
        moments_gen<R, D, M, EN, false>(pf, mo);
      }
      const R* sf = static_of(buf_of(s));
      State<R, D, M> st;
      st.template from_moments<EN, false>(p, mo, slow ? a.phi[n] : sf[0], EN ? R(0) : (slow ? a.Tfix[n] : sf[SSTR]));
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
      if (KEEP) st_new = st;
    }
    if (s + PD <= mend) {
      issue(s + PD);
      last_issued = s + PD;
    } else if (!(TMA && bulk)) {
      cp_async_commit();
    }
    if constexpr (TMA) {
      if (__syncthreads_or(!ok)) {                   // a copy never landed: stop marching
        if (t == 0) flag(a.status, kStatusTimeout);
        aborted_at = s;
        break;
      }
    } else {
      __syncthreads();
    }
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
      } else if constexpr (TMA) {
        RowPull<R, LB::CH, LB::W> pf{col_of(buf_of(y))};
        moments_gen<R, D, M, EN, true>(pf, mo);
      } else {
        SmemPull<R, D> pf{col_of(buf_of(y)), TX};
        moments_gen<R, D, M, EN, true>(pf, mo);
      }
      // this thread's ring column is its collide column (xm == xt here)
      const R* sf = static_of(buf_of(y));
      State<R, D, M> st;
      if (KEEP) st = st_prev;
      else st.template from_moments<EN, true>(p, mo, slow ? a.phi[n] : sf[0], EN ? R(0) : (slow ? a.Tfix[n] : sf[SSTR]));
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
      } else if constexpr (TMA) {
        RowPull<R, LB::CH, LB::W> pf{col_of(buf_of(y))};
        collide_gen<R, D, M, EN>(p, pf, n, mo, st, gr, a.dst, a.status);
      } else {
        SmemPull<R, D> pf{col_of(buf_of(y)), TX};
        collide_gen<R, D, M, EN>(p, pf, n, mo, st, gr, a.dst, a.status);
      }
    }
    if (KEEP) st_prev = st_new;
    __syncthreads();
  }
  if (TMA && bulk) {
    // after an abort, drain the bulk copies still in flight (bounded)
    if (aborted_at <= mend)
      for (int r = aborted_at; r <= last_issued; ++r)
        if (!mbar_wait(bar + buf_of(r), (uint32_t)(((r - (m0 - 1)) / NBUF) & 1), 1 << 20)) break;
  } else {
    cp_async_wait<0>();
  }
}

}  // namespace lbm
