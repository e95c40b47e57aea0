// Internal declarations shared by the host API and the CUDA kernels of
// liblbrt.so.  Nothing here is part of the public ABI (include/lb_rt.h).
#pragma once

#include <cuda.h>
#include <cuda_runtime.h>
#include <cuda_fp16.h>
#include <cuda_bf16.h>
#include <cudaTypedefs.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "lb_rt.h"

namespace lbrt {

// Per-direction constants handed to the kernels by value (kernel parameters
// live in the constant bank, so a warp reading the same direction gets a
// broadcast).  nw = (n_x, n_y, n_z, w); au = (a_x, a_y, a_z, octant bits),
// a = cfl |n| the weight of the upwind corner along each axis in Eq. (interp);
// octant bit k set means sgn(n_k) = -1, i.e. the pull reads the +1 neighbour
// along axis k.
// The table is in the library's internal direction order (see the planner in
// lb_rt_api.cu): directions grouped by (sgn n^y, sgn n^z), each group padded
// with inert entries (w = 0, n = 0, octant bit 3 set) whose populations stay 0.
constexpr int kMaxInternalDirs = 256;
struct DirTable {
  float4 nw[kMaxInternalDirs];
  float4 au[kMaxInternalDirs];
};

// Device layout of a population buffer: [PZ][PY][N][PX], x fastest.  The
// interior nz x ny x nx grid sits inside one ghost layer: site (x, y, z) of
// direction i is element i * si + (z + 1) * sz + (y + 1) * sy + x + GL with
// si = PX, sy = N * PX, sz = N * PX * PY.  Keeping the N rows of one (y, z)
// next to each other keeps every CTA's working set (all directions of a few
// rows) within a few contiguous megabytes instead of N blocks that are
// gigabytes apart.  GL = 2 keeps even x at even columns (8-byte pairs); PX is
// a multiple of 8 so that rows start on 16-byte boundaries (TMA strides) in
// every storage type.  Ghost cells of a periodic axis mirror the opposite
// interior edge (column 1 <- x = nx - 1, column nx + GL <- x = 0, row 0 <-
// y = ny - 1, row ny + 1 <- y = 0, plane 0 <- z = nz - 1, plane nz + 1 <- z = 0);
// on a vacuum axis they stay 0.  Every kernel that writes populations also
// writes the mirrors, so a pull from x - 1, y - 1 or z - 1 (or + 1) never
// needs boundary logic.
constexpr int GL = 2;

struct Grid {
  int nx, ny, nz;
  int dims;
  long long sites;   // nx * ny * nz
  int periodic[3];   // per axis x, y, z
  int PX, PY, PZ;    // padded extents
  long long si, sy, sz;  // element strides of direction, row and plane
  long long total;   // elements of one buffer: sz * PZ
};

__host__ __device__ inline long long pidx(const Grid& g, int i, int z, int y, int x) {
  return (long long)i * g.si + (long long)(z + 1) * g.sz + (long long)(y + 1) * g.sy + (x + GL);
}

// Site coefficient fields (dense [nz][ny][nx]): nullptr means "use the scalar".
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
  int N;               // internal direction count (padding included)
  int dpt, zc;         // tile plan of the static kernel: directions per warp, planes per batch
  int nzc, ctas;       // static kernel: z chunks per column, CTAs of the persistent grid
  float dt;
  int collision;       // LB_RT_IMPLICIT_EXACT / LB_RT_EXPLICIT / LB_RT_LAMBDA_K
  int lambda_iters;
  const void* in;      // populations at t (padded layout)
  void* out;           // populations at t + dt
  const CUtensorMap* tmap_in;  // TMA descriptor of `in` (host copy)
  const CUtensorMap* tmap_e;   // 16-bit storage: TMA descriptor of the E array at t
  const float* e_in;           // 16-bit storage: E array at t (padded, float32)
  float* e_out;                // 16-bit storage: E array at t + dt (padded, float32)
  double* budget_partials;  // [nblocks][2] (sum E*, sum E_collided) or nullptr
  long long partials_cap;   // slots available; a launcher whose grid is larger refuses
  unsigned* err;            // device error word
  float* mom_E;             // FP32 static step: E of the new state, dense [sites], or nullptr
  float* mom_F;             // FP32 static step: F of the new state, dense [3][sites], or nullptr
  bool sc;                  // static step: the pipelined kernel (kernels_sc.cu)
};

// One problem of a static step launch.  The single-problem launch passes it
// as a kernel parameter; the batched launch passes a device array of them
// (with the tensor maps in device memory) and the persistent CTAs walk the
// concatenation of all problems' tiles, tiles [tile_start, tile_start +
// ntiles) belonging to this problem.
struct ProblemDesc {
  Grid g;
  void* out;                  // populations at t + dt (padded layout)
  float* e_out;               // 16-bit storage: E array at t + dt
  const CUtensorMap* tmap;    // TMA descriptor of the populations at t (batched launch)
  const CUtensorMap* emap;    // 16-bit storage: TMA descriptor of the E array at t
  StaticCoef cf;
  float dt;
  int collision, lambda_iters;
  int nzc;                    // z chunks per column of tiles
  int tile_start, ntiles;
  double* budget_partials;    // single-problem launch only
  float* mom_E;               // single-problem FP32 launch: E of the new state [sites] or nullptr
  float* mom_F;               // single-problem FP32 launch: F of the new state [3][sites] or nullptr
};

// A batched static step: every problem of `table` (device memory) has the
// same internal direction table, plan and storage.
struct BatchLaunch {
  const ProblemDesc* table;  // device array
  int nprob, ntiles;         // problems, total tiles
  int N, dpt, zc, storage;
  int ctas;
  int periodic;              // some problem has a periodic axis
  int alt;                   // 1: the alternative batched kernel of this dpt (batch_alt_zc)
  unsigned* err;
};
cudaError_t launch_tma_static_batch(const BatchLaunch& B, const DirTable& t, cudaStream_t s);
cudaError_t launch_tma16_static_batch(const BatchLaunch& B, const DirTable& t, cudaStream_t s);
cudaError_t occupancy_static_batch(int storage, int dpt, int zc, int G, int* per_sm, int alt = 0);
// Planes per batch of the alternative batched kernel compiled for this storage
// and directions-per-warp (same memory layout, other registers / planes per
// batch, timed by the batch autotuner against the tile plan's own kernel), or
// 0 when there is none.
int batch_alt_zc(int storage, int dpt);
int batch_alt_zc16(int dpt);
// Two groups with different tile plans in ONE batched launch: group A's
// problems run on CTAs 0 .. ctas_a - 1 of the ctas-CTA grid, group B's on the
// rest; a block has the warps of the larger plan.  Supported for the plan
// pairs each storage type compiles (static_batch_pair_supported); A and B in
// that pair's order.
bool static_batch_pair_supported(int storage, int dpt_a, int zc_a, int dpt_b, int zc_b);
cudaError_t launch_static_batch_pair(const BatchLaunch& A, const DirTable& ta, const BatchLaunch& B,
                                     const DirTable& tb, int ctas_a, int ctas, cudaStream_t s);
cudaError_t occupancy_static_batch_pair(int storage, int dpt_a, int zc_a, int ga, int dpt_b,
                                        int zc_b, int gb, int* per_sm);
bool tma16_pair_supported(int da, int za, int db, int zb);
cudaError_t launch_tma16_static_batch_pair(const BatchLaunch& A, const DirTable& ta,
                                           const BatchLaunch& B, const DirTable& tb, int ctas_a,
                                           int ctas, cudaStream_t s);
cudaError_t occupancy_tma16_pair(int storage, int da, int za, int ga, int db, int zb, int gb,
                                 int* per_sm);

// Kernel launchers.  Return cudaGetLastError() (or an error without
// launching when the configuration is not supported).
cudaError_t launch_step_static(const StepLaunch& L, const StaticCoef& c, const DirTable& t,
                               int storage, cudaStream_t s, int* nblocks);
cudaError_t launch_step_moving(const StepLaunch& L, const MovingCoef& c, const DirTable& t,
                               int storage, cudaStream_t s, int* nblocks);
// Ni = internal direction count; Next = external (user) count; int_of_ext =
// device array mapping an external direction index to its internal one.
// e = the padded float32 E array paired with `pop` (16-bit storage only).
cudaError_t launch_moments(const Grid& g, int Ni, const void* pop, const float* e, int storage,
                           const DirTable& t, float* E, float* F, float* P, cudaStream_t s);
cudaError_t launch_init_state(const Grid& g, int Ni, int Next, const int* int_of_ext,
                              const float* data, int kind, void* pop, float* e, int storage,
                              const DirTable& t, cudaStream_t s);
cudaError_t launch_decode(const Grid& g, int Next, const int* int_of_ext, const void* pop,
                          const float* e, int storage, const DirTable& t, float* out,
                          cudaStream_t s);
cudaError_t launch_frozen(const Grid& g, int Ni, int Next, const int* int_of_ext, int ncells,
                          const int64_t* cells, const float* vals, void* pop, float* e,
                          int storage, const DirTable& t, double* injection_acc, cudaStream_t s);
cudaError_t launch_budget_finalize(const double* partials, int nblocks, double* acc,
                                   cudaStream_t s);
// Coupling outputs J [sites], H [3][sites], S [4][sites] (any may be null).
cudaError_t launch_coupling(const Grid& g, int N, const void* pop, const float* e, int storage,
                            const DirTable& t, const MovingCoef& c, float* J, float* H, float* S,
                            cudaStream_t s);
cudaError_t launch_total_energy(const Grid& g, int N, const void* pop, const float* e, int storage,
                                const DirTable& t, double* partials, int max_blocks, double* out,
                                cudaStream_t s);

// TMA descriptor of a padded float32 population buffer viewed as the 4D
// tensor [PZ][PY][Ni][PX] with box (68, dpt, 2, zc) (kernels_tma.cu), and the
// tile plans the static kernel is compiled for.
bool make_pop_tensor_map(CUtensorMap* map, const Grid& g, int Ni, void* base, int dpt, int zc,
                         std::string& err);
extern const int kTilePlans[][3];
extern const int kNumTilePlans;
size_t step_tile_smem(int dpt, int zc, int warps);
// z chunks and CTA count of the static kernel's persistent grid for this
// grid and plan on the current device (occupancy query).
cudaError_t plan_static_grid(const Grid& g, int Ni, int dpt, int zc, int storage, int* nzc,
                             int* ctas, bool moving = false, bool sc = false);
// Moving fluid, FP32 populations, TMA tiles (kernels_tma_moving.cu): one
// plane per batch; plans (directions per warp, 1, thread cap).
extern const int kTilePlansMoving[][3];
extern const int kNumTilePlansMoving;
size_t step_tile_smem_moving(int dpt, int warps);
cudaError_t occupancy_tma_moving(int dpt, int G, int* per_sm);
cudaError_t launch_tma_moving(const StepLaunch& L, const MovingCoef& c, const DirTable& t,
                              cudaStream_t s, int* nblocks);
cudaError_t occupancy_tma16_moving(int storage, int dpt, int G, int* per_sm);
cudaError_t launch_tma16_moving(const StepLaunch& L, const MovingCoef& c, const DirTable& t,
                                int storage, cudaStream_t s, int* nblocks);
// Pipelined static step (kernels_sc.cu), float32 and 16-bit storage, single
// problem: plans (directions per warp, planes per batch, thread cap with the
// coefficient warps); shared memory and resident CTAs per SM for
// `stream_warps` stream warps.
extern const int kTilePlansSC[][3];
extern const int kNumTilePlansSC;
size_t step_tile_smem_sc(int storage, int dpt, int zc, int stream_warps);
cudaError_t occupancy_sc(int storage, int dpt, int zc, int stream_warps, int* per_sm);
cudaError_t launch_sc_static(const StepLaunch& L, const StaticCoef& c, const DirTable& t, int storage,
                             cudaStream_t s, int* nblocks);
// 16-bit storage (kernels_tma16.cu): f_i = I_i / w_i = E (1 + q_i) with E a
// padded float32 [PZ][PY][PX] array and q_i stored in FP16 or BF16.
size_t step_tile_smem16(int dpt, int zc, int warps);
extern const int kTilePlans16[][3];
extern const int kNumTilePlans16;
cudaError_t launch_tma16_static(const StepLaunch& L, const StaticCoef& c, const DirTable& t,
                                int storage, cudaStream_t s, int* nblocks);
cudaError_t occupancy_tma16(int storage, int dpt, int zc, int G, int* per_sm, bool batch = false,
                            int alt = 0);
bool make_pop16_tensor_map(CUtensorMap* map, const Grid& g, int Ni, void* base, int storage, int dpt,
                           int zc, std::string& err);
bool make_e_tensor_map(CUtensorMap* map, const Grid& g, float* base, int zc, std::string& err);
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder(std::string& err);

// Message returned by lb_rt_last_error(NULL) on this thread (calls without a handle).
void set_unbound_error(const std::string& m);

// Direction sets built on the host (directions.cpp).
bool build_directions(const lb_rt_config& cfg, std::vector<double>& n, std::vector<double>& w,
                      std::string& err);

// ---- device helpers shared by the kernels --------------------------------

// Padded positions mirroring interior coordinate c of an axis of extent n:
// the own position and, on a periodic axis, the ghost on the opposite side.
__device__ __forceinline__ int mirrors(int c, int n, int periodic, int off, int* out) {
  int m = 0;
  out[m++] = c + off;
  if (periodic) {
    if (c == n - 1) out[m++] = off - 1;
    if (c == 0) out[m++] = n + off;
  }
  return m;
}

// Store one population value at site (x, y, z) of direction i and at every
// ghost mirror of that site on the periodic axes.
template <class T>
__device__ __forceinline__ void store_pop(T* pop, const Grid& g, int i, int z, int y, int x,
                                          T v) {
  int xs[3], ys[3], zs[3];
  const int nxs = mirrors(x, g.nx, g.periodic[0], GL, xs);
  const int nys = mirrors(y, g.ny, g.periodic[1], 1, ys);
  const int nzs = mirrors(z, g.nz, g.periodic[2], 1, zs);
  const long long base = (long long)i * g.si;
  for (int a = 0; a < nzs; ++a)
    for (int b = 0; b < nys; ++b)
      for (int c = 0; c < nxs; ++c)
        pop[base + (long long)zs[a] * g.sz + (long long)ys[b] * g.sy + xs[c]] = v;
}

// True when site (x, y, z) has at least one ghost mirror.
__device__ __forceinline__ bool has_mirror(const Grid& g, int z, int y, int x) {
  return (g.periodic[0] && (x == 0 || x == g.nx - 1)) ||
         (g.periodic[1] && (y == 0 || y == g.ny - 1)) ||
         (g.periodic[2] && (z == 0 || z == g.nz - 1));
}

}  // namespace lbrt
