// Internal: the library context behind the opaque lbm_ctx handle.
#pragma once

#include <cuda_runtime.h>

#include <string>
#include <vector>

#include "../../include/lbm.h"
#include "lbm_batch.cuh"
#include "lbm_kernels.cuh"
#include "lbm_ops.h"
#include "lbm_surface.cuh"

struct lbm_ctx {
  int nx, ny, nz, N, D, Q, M, L, energy, knudsen, precision, S;
  double dt, cvel;
  cudaStream_t stream;
  void* pops[2];
  int cur;
  void* phi;
  void* Tfix;
  void* mac;
  int* status;
  double* scratch_out;        // device buffer for lbm_moments to host
  size_t scratch_bytes;
  lbm::Params<double> pd;
  lbm::Params<float> pf;
  lbm::InletTables<double> itd;
  lbm::InletTables<float> itf;
  lbm::Ops<double> od;
  lbm::Ops<float> of;
  std::string err;
  // kernel timing (lbm_set_timing)
  int timing;
  std::vector<cudaEvent_t> ev;       // start/stop pairs
  std::vector<int> ev_kind;
  size_t ev_used;
  int variant;                       // < 0: two-pass form; >= 0: fused tile shape
  long long steps_done;              // steps taken through lbm_step (checkpoint images carry it)
  // streaming steps on host-resident states (lbm_step_host): two pairs of
  // device state slots used by alternate calls, an upload and a download
  // stream, and per pair the events ordering upload -> steps -> download
  void* hslot[4];
  cudaStream_t h2d, d2h;
  cudaEvent_t ev_in[2], ev_done[2], ev_free[2];
  bool free_recorded[2];
  long long hcall;
  // surface mechanism (S > 0): coverages (ping-pong), per-node sources, mechanism table
  double* Xs[2];
  int xs_cur;
  double* rsrc;
  double* dphi_dev;                  // per-node potential difference of the TPB steps (lbm_set_potential)
  lbm::MechDev* mech;
  // initial fields kept on the device (lbm_adjoint restarts from them)
  double* init_X;                    // [M][N]
  double* init_T;                    // [N]
  double* init_P;                    // [N]
  double* init_U;                    // [3][N] or null
  double tortuosity, pore_radius;
  // batched form (lbm_create_batch; n_cases == 0 for a single lattice)
  int n_cases;
  std::vector<int> case_N, case_nx, case_ny;
  std::vector<long long> case_node_off;
  std::vector<double> case_dt, case_cvel;
  std::vector<lbm::Params<double>> case_pd;
  std::vector<lbm::Params<float>> case_pf;
  std::vector<lbm::InletTables<double>> case_itd;
  std::vector<lbm::InletTables<float>> case_itf;
  void* cases_dev;                   // CaseDev<R>[n_cases]
  int2* tiles_dev[3];                // work lists for tile lengths 64, 128, 256
  int ntiles[3];
  lbm::BatchOps<double> bd;
  lbm::BatchOps<float> bf;
  int sm_count;
  cudaStream_t cap_stream;           // private stream for graph capture
  cudaGraphExec_t gexec[2];          // 50-step graphs for each ping-pong parity
  int gvariant[2];
};

namespace lbm {
// lattice-unit parameters of a validated configuration (lbm_capi.cu)
void make_params(const lbm_config* c, Params<double>& p, InletTables<double>& it, double& dt, double& cvel);
}
