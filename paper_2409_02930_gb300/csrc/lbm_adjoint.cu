// Host side of lbm_adjoint: forward run with checkpoints, segment-wise
// recomputation and the reverse sweep of the adjoint kernels.
#include <cuda_runtime.h>

#include <cstring>
#include <string>
#include <vector>

#include "lbm_adjoint.cuh"
#include "lbm_ctx.h"

namespace {

const double R_UNIV_SI_ADJ = 8.314462618;   // J/(mol K)

int adj_fail(lbm_ctx* x, int code, const std::string& msg) {
  x->err = msg;
  return code;
}

// Device buffers of one lbm_adjoint call, freed on every exit path.
struct Scratch {
  std::vector<void*> ptrs;
  ~Scratch() {
    for (void* p : ptrs) cudaFree(p);
  }
  template <class T>
  cudaError_t alloc(T** out, size_t bytes) {
    void* p = nullptr;
    cudaError_t e = cudaMalloc(&p, bytes);
    if (e == cudaSuccess) ptrs.push_back(p);
    *out = (T*)p;
    return e;
  }
};

template <class B>
int run_adjoint(lbm_ctx* x, const lbm::Ops<B>& ops, const lbm::Params<B>& p, const lbm::InletTables<B>& it,
                const lbm::AdjOps<B>& adj, const lbm_objective* obj, int n_steps, int C, double* J_out,
                double* dJ_dphi, double* dJ_dpore, double* dJ_dtort) {
  const size_t N = x->N;
  const size_t LQN = (size_t)x->L * x->Q * N;
  const size_t state = LQN * sizeof(B);
  const int nck = n_steps > 0 ? (n_steps + C - 1) / C : 0;
  cudaStream_t s = x->stream;
  Scratch sc;
  B *ck = nullptr, *seg = nullptr, *lamA = nullptr, *lamB = nullptr, *Pbar = nullptr, *Gbar = nullptr;
  double *phibar = nullptr, *kbar = nullptr, *jbuf = nullptr;
  cudaError_t e = sc.alloc(&ck, state * (nck > 0 ? nck : 1));
  if (e == cudaSuccess) e = sc.alloc(&seg, state * (C > 1 ? C - 1 : 1));
  if (e == cudaSuccess) e = sc.alloc(&lamA, state);
  if (e == cudaSuccess) e = sc.alloc(&lamB, state);
  if (e == cudaSuccess) e = sc.alloc(&Pbar, state);
  if (e == cudaSuccess) e = sc.alloc(&Gbar, (size_t)adj.n_grad * N * sizeof(B));
  if (e == cudaSuccess) e = sc.alloc(&phibar, N * sizeof(double));
  if (e == cudaSuccess) e = sc.alloc(&kbar, N * sizeof(double));
  if (e == cudaSuccess) e = sc.alloc(&jbuf, (size_t)x->M * x->D * N * sizeof(double));
  if (e != cudaSuccess) return adj_fail(x, LBM_ERR_ALLOC, "adjoint scratch allocation failed");
  B* mac = (B*)x->mac;
  const B* phi = (const B*)x->phi;
  const B* Tfix = (const B*)x->Tfix;
  // forward and recompute steps in the context's kernel form
  auto step = [&](const B* src, B* dst) {
    lbm::StepArgs<B> a{src, dst, phi, Tfix, mac, x->status};
    if (x->variant >= 0 && ops.fused(p, it, a, x->variant, s) == 0) return;
    ops.macro(p, it, a, s);
    ops.collide(p, it, a, s);
  };
  // ---- forward run from the initial equilibria, with checkpoints ---------
  cudaMemsetAsync(x->status, 0, sizeof(int), s);
  x->cur = 0;
  B* cur = (B*)x->pops[0];
  B* nxt = (B*)x->pops[1];
  ops.init(p, x->init_X, x->init_T, x->init_P, x->init_U, x->cvel, R_UNIV_SI_ADJ, cur, phi, s);
  for (int k = 0; k < n_steps; ++k) {
    if (k % C == 0) cudaMemcpyAsync(ck + (size_t)(k / C) * LQN, cur, state, cudaMemcpyDeviceToDevice, s);
    step(cur, nxt);
    B* t = cur;
    cur = nxt;
    nxt = t;
    x->cur = 1 - x->cur;
  }
  // ---- objective on the final state ----------------------------------------
  {
    lbm::StepArgs<B> a{cur, nullptr, phi, Tfix, mac, x->status};
    ops.moments(p, it, a, LBM_MOM_J_A, x->cvel, jbuf, s);
    std::vector<double> j((size_t)x->M * x->D * N);
    e = cudaMemcpyAsync(j.data(), jbuf, j.size() * sizeof(double), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) return adj_fail(x, LBM_ERR_CUDA, std::string("adjoint forward: ") + cudaGetErrorString(e));
    int st = 0;
    cudaMemcpy(&st, x->status, sizeof(int), cudaMemcpyDeviceToHost);
    if (st & 1) return adj_fail(x, LBM_ERR_NUMERIC, "non-finite state in the forward run");
    double J = 0.0;
    const double* ja = j.data() + ((size_t)obj->species * x->D + obj->axis) * N;
    for (size_t n = obj->plane; n < N; n += x->nx) J += ja[n];
    if (J_out) *J_out = obj->weight * J;
  }
  // ---- adjoint of the final state ---------------------------------------------
  cudaMemsetAsync(phibar, 0, N * sizeof(double), s);
  cudaMemsetAsync(kbar, 0, N * sizeof(double), s);
  lbm::AdjArgs<B> a{cur, mac, phi, Tfix, nullptr, Pbar, Gbar, phibar, kbar, lamA, x->status};
  adj.seed_flux(p, a, obj->species, obj->axis, obj->plane, obj->weight, s);
  const bool inlet = (p.bc_lo == lbm::BC_INLET) || (p.bc_hi == lbm::BC_INLET);
  if (inlet && adj.ghost(p, it, a, s)) return adj_fail(x, LBM_ERR_CUDA, "adjoint ghost launch");
  adj.stream(p, a, s);
  B* lam1 = lamA;     // adjoint of f^{k+1}
  B* lam0 = lamB;
  // ---- reverse sweep, one checkpoint segment at a time ---------------------
  for (int sg = nck - 1; sg >= 0; --sg) {
    const int k0 = sg * C, k1 = (k0 + C < n_steps) ? k0 + C : n_steps;
    const B* base = ck + (size_t)sg * LQN;
    auto state_of = [&](int k) -> const B* { return k == k0 ? base : seg + (size_t)(k - k0 - 1) * LQN; };
    for (int k = k0; k + 1 < k1; ++k) step(state_of(k), seg + (size_t)(k - k0) * LQN);
    for (int k = k1 - 1; k >= k0; --k) {
      const B* f = state_of(k);
      lbm::StepArgs<B> sa{f, nullptr, phi, Tfix, mac, x->status};
      ops.macro(p, it, sa, s);
      lbm::AdjArgs<B> aa{f, mac, phi, Tfix, lam1, Pbar, Gbar, phibar, kbar, lam0, x->status};
      if (adj.collide(p, it, aa, s) || adj.macro(p, it, aa, s) || (inlet && adj.ghost(p, it, aa, s)))
        return adj_fail(x, LBM_ERR_CUDA, "adjoint kernel launch");
      adj.stream(p, aa, s);
      B* t = lam1;
      lam1 = lam0;
      lam0 = t;
    }
  }
  // ---- initial equilibria ------------------------------------------------------
  {
    lbm::AdjArgs<B> aa{nullptr, mac, phi, Tfix, nullptr, Pbar, Gbar, phibar, kbar, lam1, x->status};
    adj.init(p, x->init_X, x->init_T, x->init_P, x->init_U, x->cvel, R_UNIV_SI_ADJ, aa, s);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return adj_fail(x, LBM_ERR_CUDA, std::string("adjoint: ") + cudaGetErrorString(e));
  std::vector<double> kb(N);
  if (dJ_dphi) e = cudaMemcpyAsync(dJ_dphi, phibar, N * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaMemcpyAsync(kb.data(), kbar, N * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) return adj_fail(x, LBM_ERR_CUDA, std::string("adjoint: ") + cudaGetErrorString(e));
  double dl = 0.0;
  for (size_t n = 0; n < N; ++n) dl += kb[n];
  // 1/tau^k is proportional to tortuosity / pore radius: d/dlambda = tau d/dtau = -r_p d/dr_p
  if (dJ_dtort) *dJ_dtort = x->knudsen ? dl / x->tortuosity : 0.0;
  if (dJ_dpore) *dJ_dpore = x->knudsen ? -dl / x->pore_radius : 0.0;
  int st = 0;
  cudaMemcpy(&st, x->status, sizeof(int), cudaMemcpyDeviceToHost);
  if (st & 1) return adj_fail(x, LBM_ERR_NUMERIC, "non-finite value in the adjoint sweep");
  return LBM_OK;
}

}  // namespace

extern "C" int lbm_adjoint(lbm_ctx* x, const lbm_objective* obj, int n_steps, int ckpt_every, double* J,
                           double* dJ_dphi, double* dJ_dpore, double* dJ_dtort) {
  if (!x) return LBM_ERR_ARG;
  if (!obj || obj->kind != LBM_OBJ_PLANE_FLUX) return adj_fail(x, LBM_ERR_ARG, "unknown objective");
  if (n_steps < 0 || ckpt_every < 1) return adj_fail(x, LBM_ERR_ARG, "n_steps < 0 or ckpt_every < 1");
  if (x->n_cases > 0 || x->S > 0 || x->D != 2)
    return adj_fail(x, LBM_ERR_ARG, "the adjoint supports single 2-D lattices without surface mechanism");
  if (obj->species < 0 || obj->species >= x->M || obj->axis < 0 || obj->axis >= x->D || obj->plane < 0 ||
      obj->plane >= x->nx)
    return adj_fail(x, LBM_ERR_ARG, "objective species, axis or plane out of range");
  if (x->precision == LBM_FP64) {
    lbm::AdjOps<double> adj;
    if (!lbm::get_adj_ops_f64(x->D, x->M, x->energy, &adj))
      return adj_fail(x, LBM_ERR_ARG, "no adjoint kernels for this (M, energy)");
    return run_adjoint(x, x->od, x->pd, x->itd, adj, obj, n_steps, ckpt_every, J, dJ_dphi, dJ_dpore, dJ_dtort);
  }
  lbm::AdjOps<float> adj;
  if (!lbm::get_adj_ops_f32(x->D, x->M, x->energy, &adj))
    return adj_fail(x, LBM_ERR_ARG, "no adjoint kernels for this (M, energy)");
  return run_adjoint(x, x->of, x->pf, x->itf, adj, obj, n_steps, ckpt_every, J, dJ_dphi, dJ_dpore, dJ_dtort);
}
