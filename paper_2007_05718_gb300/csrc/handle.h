// The opaque handle of include/lb_rt.h, shared by the host API (lb_rt_api.cu)
// and the batch runtime (batch.cu).  Not part of the public ABI.
#pragma once

#include <string>
#include <vector>

#include "lb_rt_internal.h"

struct lb_rt {
  using Grid = lbrt::Grid;
  using DirTable = lbrt::DirTable;
  using StaticCoef = lbrt::StaticCoef;
  using MovingCoef = lbrt::MovingCoef;
  lb_rt_config cfg{};
  Grid grid{};
  int N = 0;                    // directions, external (user) order
  int Ni = 0;                   // internal directions including inert padding
  int dpt = 0, zc = 0;          // tile plan of the static kernel
  bool pipelined = false;       // single-problem static steps run the pipelined kernel
  int nzc = 0, ctas = 0;        // its persistent grid: z chunks, CTAs
  std::vector<int> ext_of_int;  // internal -> external index (-1: padding)
  std::vector<int> int_of_ext;  // external -> internal index
  int* d_int_of_ext = nullptr;  // device copy
  double dt = 0.0;
  std::vector<double> n, w;
  DirTable table{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int device = 0;
  void* pop[2] = {nullptr, nullptr};
  float* ef[2] = {nullptr, nullptr};   // 16-bit storage: padded E arrays paired with pop[]
  size_t ef_bytes = 0;
  CUtensorMap tmap[2];                 // TMA descriptors of pop[0] / pop[1]
  CUtensorMap emap[2];                 // 16-bit storage: TMA descriptors of ef[0] / ef[1]
  bool tmap_ok = false;
  bool iso = false;             // isotropic table: sum w = 1, sum w n = 0, sum w n n = Id / d
  int cur = 0;
  size_t pop_bytes = 0;
  // coefficient fields: static ka, k0, lam, eta (slots 0-3); moving v(3), kta, kt0, etat (4-7)
  float* fld[8] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};
  StaticCoef sc{};
  MovingCoef mc{};
  int64_t* frozen_cells = nullptr;
  float* frozen_vals = nullptr;
  int nfrozen = 0;
  double* partials = nullptr;
  int partials_cap = 0;
  double* acc = nullptr;       // 8 doubles, see k_budget_finalize
  unsigned* err = nullptr;     // device error word
  unsigned* err_host = nullptr;  // page-locked host copy of it, read after each sync
  float* scratch = nullptr;    // moments staging for host outputs [10][sites]
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  bool timing = false;
  float last_ms = 0.f;
  int last_nlaunch = 0;
  long long steps = 0;
  std::string msg;
};

// Internal entry points of lb_rt_api.cu used by the batch runtime.
namespace lbrt {
// Bytes of device memory lb_rt_create() would allocate for `cfg` (estimate
// from the padded layout and the planner, without touching the device).
size_t handle_device_bytes(const lb_rt_config& cfg, std::string& err);
}  // namespace lbrt
