// Internal declarations shared by the host API and the CUDA kernels of
// liblbrt.so.  Nothing here is part of the public ABI (include/lb_rt.h).
#pragma once

#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lb_rt.h"

namespace lbrt {

// Per-direction constants handed to the step kernels by value (kernel
// parameters live in the constant bank, so a warp reading the same
// direction gets a broadcast).  nw = (n_x, n_y, n_z, w);
// au = (a_x, a_y, a_z, upwind octant bits) with a = cfl |n| the weight of
// the upwind corner along each axis in Eq. (interp); octant bit k set means
// sgn(n_k) = -1, i.e. the pull reads the +1 neighbour along axis k.
struct DirTable {
  float4 nw[LB_RT_MAX_DIRS];
  float4 au[LB_RT_MAX_DIRS];
};

// Geometry and boundary data of one grid.
struct Grid {
  int nx, ny, nz;
  int dims;
  long long sites;   // nx * ny * nz
  int periodic[3];   // per axis x, y, z
};

// Site coefficient fields: pointer == nullptr means "use the scalar".
struct StaticCoef {
  const float* ka; const float* k0; const float* lam; const float* eta;
  float ka_s, k0_s, lam_s, eta_s;
};

struct MovingCoef {
  const float* v;    // [3][sites] or nullptr (fluid at rest)
  const float* kta; const float* kt0; const float* etat;
  float kta_s, kt0_s, etat_s;
};

enum StorageKind { ST_F32 = 0, ST_F16 = 1, ST_BF16 = 2 };

struct StepLaunch {
  Grid g;
  int N;
  float dt;
  int collision;       // LB_RT_IMPLICIT_EXACT / LB_RT_EXPLICIT / LB_RT_LAMBDA_K
  int lambda_iters;
  const void* in;      // populations at t
  void* out;           // populations at t + dt
  const float4* ef_in; // per-site moments of `in` (reduced-precision modes)
  float4* ef_out;
  double* budget_partials;  // [nblocks][2] (sum E*, sum E_collided) or nullptr
  unsigned* err;            // device error word
};

// Kernel launchers (kernels_*.cu).  Return cudaGetLastError().
cudaError_t launch_step_static(const StepLaunch& L, const StaticCoef& c, const DirTable& t,
                               int storage, cudaStream_t s, int* nblocks);
cudaError_t launch_step_moving(const StepLaunch& L, const MovingCoef& c, const DirTable& t,
                               int storage, cudaStream_t s, int* nblocks);
cudaError_t launch_moments(const Grid& g, int N, const void* pop, const float4* ef, int storage,
                           const DirTable& t, float* E, float* F, float* P, cudaStream_t s);
cudaError_t launch_init_state(const Grid& g, int N, const float* data, int kind, void* pop,
                              float4* ef, int storage, const DirTable& t, cudaStream_t s);
cudaError_t launch_decode(const Grid& g, int N, const void* pop, const float4* ef, int storage,
                          const DirTable& t, float* out, cudaStream_t s);
cudaError_t launch_frozen(const Grid& g, int N, int ncells, const int64_t* cells, const float* vals,
                          void* pop, float4* ef, int storage, const DirTable& t,
                          double* injection_acc, cudaStream_t s);
cudaError_t launch_budget_finalize(const double* partials, int nblocks, double* acc,
                                   cudaStream_t s);
cudaError_t launch_total_energy(const Grid& g, int N, const void* pop, const float4* ef,
                                int storage, const DirTable& t, double* partials, int max_blocks,
                                double* out, cudaStream_t s);

// Direction sets built on the host (directions.cpp).
bool build_directions(const lb_rt_config& cfg, std::vector<double>& n, std::vector<double>& w,
                      std::string& err);

}  // namespace lbrt
