// Scratch-free time step (lbm_step_noalloc in include/lbm.h).
//
// Some callers cannot allocate device memory while they run: a host framework
// that owns every device byte through its own pool allocator, or a
// time-critical loop in which a cudaMalloc / cudaFree (which can synchronise
// the whole device) is not acceptable.  This entry point performs one
// two-pass time step of a D2Q9 lattice whose state the caller owns, and keeps
// the only scratch the step needs -- the macro fields u, Pi and Y_a that the
// second pass reads for its gradients, plus a status word -- in a fixed-size
// array compiled into the library.  Nothing is allocated per call.
//
// The array is a file-scope __device__ object: every GPU that loads the
// library holds it (kScratchBytes) until the process exits.  Host code may
// not use the array's name as a device address; its device address is looked
// up once per device with cudaGetSymbolAddress on the first call made while
// that device is current, and reused afterwards.  All calls share the array
// and it keeps the contents of the last call, so calls whose work overlaps on
// the GPU (for example on two streams) race on it.  Each call waits for its
// step to finish and reports the step's status word in its return code.
#include <cuda_runtime.h>

#include <cstring>
#include <mutex>

#include "../../include/lbm.h"
#include "lbm_kernels.cuh"

namespace lbm {
void make_params(const lbm_config* c, Params<double>& p, InletTables<double>& it, double& dt, double& cvel);
int validate_config(const lbm_config* c);
}

namespace {

constexpr size_t kScratchBytes = 32u << 20;   // 32 MiB
constexpr size_t kStatusBytes = 256;          // status word, then the macro fields
constexpr int kMaxDevices = 64;

__device__ __align__(256) unsigned char g_step_scratch[kScratchBytes];

std::mutex g_setup_mutex;
unsigned char* g_scratch_addr[kMaxDevices] = {};

// Device address of the scratch array on the current device, looked up once
// per device (the first call made while that device is current) and reused.
// A device reset (cudaDeviceReset) unloads the library's module, so the
// cached address is no longer valid after one; callers that reset a device
// must not call this entry point again in the same process.
int scratch_address(unsigned char** out) {
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return LBM_ERR_CUDA;
  std::lock_guard<std::mutex> lock(g_setup_mutex);
  if (!g_scratch_addr[dev]) {
    void* ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_step_scratch) != cudaSuccess || !ptr) return LBM_ERR_CUDA;
    g_scratch_addr[dev] = static_cast<unsigned char*>(ptr);
  }
  *out = g_scratch_addr[dev];
  return LBM_OK;
}

template <class R>
void to_precision(const lbm::Params<double>& d, lbm::Params<R>& r, const lbm::InletTables<double>& di,
                  lbm::InletTables<R>& ri) {
  r.nx = d.nx; r.ny = d.ny; r.nz = d.nz; r.N = d.N;
  r.bc_lo = d.bc_lo; r.bc_hi = d.bc_hi; r.knudsen = d.knudsen;
  r.RU = (R)d.RU;
  for (int a = 0; a < lbm::MMAX; ++a) {
    r.m[a] = (R)d.m[a]; r.Ra[a] = (R)d.Ra[a]; r.muref[a] = (R)d.muref[a];
    r.cvR[a] = (R)d.cvR[a]; r.U0[a] = (R)d.U0[a]; r.knc[a] = (R)d.knc[a];
    for (int b = 0; b < lbm::MMAX; ++b) r.invDmm[a][b] = (R)d.invDmm[a][b];
    r.rho_in[0][a] = (R)d.rho_in[0][a]; r.rho_in[1][a] = (R)d.rho_in[1][a];
  }
  r.mu_exp = (R)d.mu_exp; r.inv_Pr = (R)d.inv_Pr; r.bulk_ratio = (R)d.bulk_ratio;
  r.T_thermo = (R)d.T_thermo; r.inv_T_ref = (R)d.inv_T_ref; r.Pref = (R)d.Pref;
  r.T_in[0] = (R)d.T_in[0]; r.T_in[1] = (R)d.T_in[1];
  r.kappa_thr = (R)d.kappa_thr;
  r.wait_limit = d.wait_limit;
  for (int s = 0; s < 2; ++s) {
    for (int a = 0; a < lbm::MMAX; ++a) ri.rho[s][a] = (R)di.rho[s][a];
    ri.rho_sum[s] = (R)di.rho_sum[s]; ri.Rmix[s] = (R)di.Rmix[s]; ri.Umix[s] = (R)di.Umix[s]; ri.T[s] = (R)di.T[s];
  }
}

template <class R, int M, bool EN>
void launch(const lbm::Params<R>& p, const lbm::InletTables<R>& it, const lbm::StepArgs<R>& a, cudaStream_t s) {
  const int grid = (p.N + 255) / 256;
  lbm::k_macro<R, 2, M, EN><<<grid, 256, 0, s>>>(p, it, a);
  lbm::k_collide<R, 2, M, EN><<<grid, 256, 0, s>>>(p, it, a);
}

template <class R>
int run(const lbm_config* c, const void* pops_in, void* pops_out, const void* porosity, const void* T_fixed,
        unsigned char* scratch) {
  lbm::Params<double> pd;
  lbm::InletTables<double> itd;
  double dt, cvel;
  lbm::make_params(c, pd, itd, dt, cvel);
  lbm::Params<R> p;
  lbm::InletTables<R> it;
  to_precision(pd, p, itd, it);
  cudaStream_t s = (cudaStream_t)c->stream;
  int* status = reinterpret_cast<int*>(scratch);
  R* mac = reinterpret_cast<R*>(scratch + kStatusBytes);
  // the status word must start at zero for every call; the macro fields are
  // overwritten by the first pass before the second pass reads them
  if (cudaMemsetAsync(status, 0, kStatusBytes, s) != cudaSuccess) return LBM_ERR_CUDA;
  lbm::StepArgs<R> a{(const R*)pops_in, (R*)pops_out, (const R*)porosity, (const R*)T_fixed, mac, status};
  const bool en = c->energy != 0;
  switch (c->M * 2 + (en ? 1 : 0)) {
    case 4: launch<R, 2, false>(p, it, a, s); break;
    case 5: launch<R, 2, true>(p, it, a, s); break;
    case 6: launch<R, 3, false>(p, it, a, s); break;
    case 7: launch<R, 3, true>(p, it, a, s); break;
    default: return LBM_ERR_ARG;
  }
  if (cudaGetLastError() != cudaSuccess) return LBM_ERR_CUDA;
  // the step's status word: bit 0 marks a non-finite or non-positive state
  int st = 0;
  if (cudaMemcpyAsync(&st, status, sizeof(int), cudaMemcpyDeviceToHost, s) != cudaSuccess) return LBM_ERR_CUDA;
  if (cudaStreamSynchronize(s) != cudaSuccess) return LBM_ERR_CUDA;
  return (st & 1) ? LBM_ERR_NUMERIC : LBM_OK;
}

}  // namespace

extern "C" {

size_t lbm_noalloc_scratch_limit(void) { return kScratchBytes - kStatusBytes; }

int lbm_step_noalloc(const lbm_config* c, const void* pops_in, void* pops_out, const void* porosity,
                     const void* T_fixed) {
  if (!c || !pops_in || !pops_out || !porosity || !T_fixed || pops_in == pops_out) return LBM_ERR_ARG;
  // the checks of lbm_create that do not need its per-node input arrays
  if (lbm::validate_config(c) != LBM_OK) return LBM_ERR_ARG;
  if (c->nz != 1 || (c->M != 2 && c->M != 3) || c->S != 0) return LBM_ERR_ARG;
  const size_t rs = c->precision == LBM_FP64 ? 8 : 4;
  const size_t need = (size_t)(2 * 2 + c->M) * (size_t)c->nx * (size_t)c->ny * rs;
  if (need > lbm_noalloc_scratch_limit()) return LBM_ERR_ARG;   // lattice too large for the static scratch
  unsigned char* scratch = nullptr;
  int rc = scratch_address(&scratch);
  if (rc != LBM_OK) return rc;
  return c->precision == LBM_FP64 ? run<double>(c, pops_in, pops_out, porosity, T_fixed, scratch)
                                  : run<float>(c, pops_in, pops_out, porosity, T_fixed, scratch);
}

}  // extern "C"
