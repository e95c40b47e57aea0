// Host side of the C ABI declared in include/lb_rt.h: validation, device
// memory, the direction table handed to the kernels, and the per-step launch
// sequence (step kernel -> frozen overwrite -> FP64 budget finalisation).
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <new>

#include "handle.h"
#include "lb_rt_internal.h"

using namespace lbrt;


namespace {

thread_local std::string g_create_msg;  // message of the last failed lb_rt_create

lb_rt_status fail(lb_rt* h, lb_rt_status st, const std::string& m) {
  if (h) h->msg = m;
  return st;
}

lb_rt_status cuda_fail(lb_rt* h, cudaError_t e, const char* where) {
  std::string m = std::string(where) + ": " + cudaGetErrorString(e);
  return fail(h, e == cudaErrorMemoryAllocation ? LB_RT_ENOMEM : LB_RT_ECUDA, m);
}

#define CK(h, call)                                    \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return cuda_fail(h, e_, #call); \
  } while (0)

size_t elem_bytes(int storage) { return storage == LB_RT_F32 ? 4 : 2; }

bool isotropic_table(const std::vector<double>& n, const std::vector<double>& w, int dims,
                     std::string& why) {
  const int N = (int)w.size();
  double T0 = 0, T1[3] = {0, 0, 0}, T2[3][3] = {{0}};
  for (int i = 0; i < N; ++i) {
    T0 += w[i];
    for (int a = 0; a < 3; ++a) {
      T1[a] += w[i] * n[3 * i + a];
      for (int b = 0; b < 3; ++b) T2[a][b] += w[i] * n[3 * i + a] * n[3 * i + b];
    }
  }
  const double tol = 1e-10;
  bool ok = std::fabs(T0 - 1.0) < tol;
  for (int a = 0; a < 3; ++a) {
    ok = ok && std::fabs(T1[a]) < tol;
    for (int b = 0; b < 3; ++b) {
      double want = (a == b && a < dims) ? 1.0 / dims : 0.0;
      ok = ok && std::fabs(T2[a][b] - want) < tol;
    }
  }
  if (!ok) why = "direction table is not isotropic to rank 2 (sum w = 1, sum w n = 0, sum w n n = I/d)";
  return ok;
}

// float32 weights whose exact sum matches the FP64 sum as closely as float32
// allows: rounding each 1/N the same way would bias sum_i w_i by up to
// N/2 ulp, and that bias would act on the energy at every step.
std::vector<float> balanced_weights(const std::vector<double>& w) {
  std::vector<float> f(w.size());
  double target = 0.0, sum = 0.0;
  for (size_t i = 0; i < w.size(); ++i) {
    f[i] = (float)w[i];
    target += w[i];
    sum += (double)f[i];
  }
  for (int pass = 0; pass < 4 && sum != target; ++pass) {
    for (size_t i = 0; i < f.size() && sum != target; ++i) {
      float g = std::nextafter(f[i], sum < target ? 2.0f : -2.0f);
      double ns = sum - (double)f[i] + (double)g;
      if (std::fabs(ns - target) < std::fabs(sum - target)) {
        sum = ns;
        f[i] = g;
      }
    }
  }
  return f;
}

// Internal direction order.  Directions are grouped by their upwind (row,
// plane) class (sgn n^y, sgn n^z); inside a class by sgn n^x, then by the
// external index.  For the static TMA kernel every class is padded to a
// multiple of the plan's directions per warp with inert entries, so that a
// warp's directions share one upwind row and one plane shift and load as a
// single box.  The plan (directions per warp, planes per batch) is the one
// with the least padding among the compiled tile plans that fit in shared
// memory.  Moving-fluid handles keep the external order.
void plan_directions(lb_rt* h) {
  const int N = h->N;
  h->ext_of_int.clear();
  h->int_of_ext.assign(N, -1);
  {
    std::vector<std::vector<int>> cls(4);
    for (int e = 0; e < N; ++e) {
      const int c = (h->n[3 * e + 1] < 0 ? 1 : 0) | (h->n[3 * e + 2] < 0 ? 2 : 0);
      cls[c].push_back(e);
    }
    for (auto& c : cls)
      std::stable_sort(c.begin(), c.end(), [&](int a, int b) {
        return (h->n[3 * a] < 0) < (h->n[3 * b] < 0);
      });
    // the first plan (in the kernel's order of preference) that fits and
    // pads the direction set by at most 4 % more than the tightest plan
    // (a moving fluid with no fitting plan falls back to the one-thread-per-
    // site kernel with this ordering and no padding).  A static handle
    // prefers the pipelined kernel's plans; the plan it takes must also fit
    // the first-generation kernel, which runs the batched launches (the
    // direction grouping fixes the summation order, so a problem gives the
    // same bits on both).
    const bool f32 = h->cfg.storage == LB_RT_F32;
    const bool mov = h->cfg.moving != 0;
    const int (*old_plans)[3] = mov ? kTilePlansMoving : f32 ? kTilePlans : kTilePlans16;
    const int n_old = mov ? kNumTilePlansMoving : f32 ? kNumTilePlans : kNumTilePlans16;
    auto pad_ni = [&](int dpt) {
      int ni = 0;
      for (auto& c : cls) ni += (int)(c.size() + dpt - 1) / dpt * dpt;
      return ni;
    };
    auto old_fits = [&](int dpt, int zc) {
      for (int p = 0; p < n_old; ++p) {
        if (old_plans[p][0] != dpt || old_plans[p][1] != zc) continue;
        if (zc > 1 && zc > h->grid.nz) return false;
        const int ni = pad_ni(dpt), warps = ni / dpt;
        if (ni > kMaxInternalDirs || 32 * warps > old_plans[p][2]) return false;
        const size_t smem = mov ? step_tile_smem_moving(dpt, warps)
                            : f32 ? step_tile_smem(dpt, zc, warps) : step_tile_smem16(dpt, zc, warps);
        return smem <= 226 * 1024;
      }
      return false;
    };
    auto choose = [&](const int (*plans)[3], int nplans, bool sc) {
      std::vector<int> ni_of(nplans, -1);
      int min_ni = 1 << 30;
      for (int p = 0; p < nplans; ++p) {
        const int dpt = plans[p][0], zc = plans[p][1];
        if (!old_fits(dpt, zc)) continue;
        const int ni = pad_ni(dpt), warps = ni / dpt;
        if (sc && (32 * (warps + zc) > plans[p][2] ||
                   step_tile_smem_sc(h->cfg.storage, dpt, zc, warps) > 226 * 1024))
          continue;
        ni_of[p] = ni;
        min_ni = std::min(min_ni, ni);
      }
      for (int p = 0; p < nplans; ++p)
        if (ni_of[p] >= 0 && ni_of[p] * 100 <= min_ni * 104) return p;
      return -1;
    };
    int best = -1;
    h->pipelined = false;
    // float32 populations keep the first-generation kernel, which measured
    // faster on the 42- and 162-direction workloads; 16-bit storage takes the
    // pipelined one
    if (!mov && !f32) {
      best = choose(kTilePlansSC, kNumTilePlansSC, true);
      if (best >= 0) {
        h->pipelined = true;
        h->dpt = kTilePlansSC[best][0];
        h->zc = kTilePlansSC[best][1];
      }
    }
    if (best < 0) {
      best = choose(old_plans, n_old, false);
      h->dpt = best >= 0 ? old_plans[best][0] : 0;
      h->zc = best >= 0 ? old_plans[best][1] : 0;
    }
    for (auto& c : cls) {
      for (int e : c) h->ext_of_int.push_back(e);
      if (h->dpt)
        for (size_t k = c.size(); k % h->dpt; ++k) h->ext_of_int.push_back(-1);
    }
  }
  h->Ni = (int)h->ext_of_int.size();
  for (int i = 0; i < h->Ni; ++i)
    if (h->ext_of_int[i] >= 0) h->int_of_ext[h->ext_of_int[i]] = i;
}

void fill_table(lb_rt* h) {
  std::memset(&h->table, 0, sizeof(h->table));
  const std::vector<float> wf = balanced_weights(h->w);
  for (int i = 0; i < h->Ni; ++i) {
    const int e = h->ext_of_int[i];
    if (e < 0) {
      // inert padding entry: no weight, no direction, the class of its
      // predecessor (its slot is part of that class's group), bit 3 set
      int oct = 8;
      if (i > 0) {
        float prev;
        std::memcpy(&prev, &h->table.au[i - 1].w, sizeof(float));
        int po;
        std::memcpy(&po, &prev, sizeof(int));
        oct |= po & 6;
      }
      float octf;
      std::memcpy(&octf, &oct, sizeof(float));
      h->table.nw[i] = make_float4(0.f, 0.f, 0.f, 0.f);
      h->table.au[i] = make_float4(0.f, 0.f, 0.f, octf);
      continue;
    }
    const double* q = &h->n[3 * e];
    h->table.nw[i] = make_float4((float)q[0], (float)q[1], (float)q[2], wf[e]);
    int oct = (q[0] < 0 ? 1 : 0) | (q[1] < 0 ? 2 : 0) | (q[2] < 0 ? 4 : 0);
    float octf;
    std::memcpy(&octf, &oct, sizeof(float));
    h->table.au[i] = make_float4((float)(h->cfg.cfl * std::fabs(q[0])),
                                 (float)(h->cfg.cfl * std::fabs(q[1])),
                                 (float)(h->cfg.cfl * std::fabs(q[2])), octf);
  }
}

lb_rt_status copy_in(lb_rt* h, void* dst, const void* src, size_t bytes, int ptr_kind) {
  if (ptr_kind != LB_RT_HOST && ptr_kind != LB_RT_DEVICE)
    return fail(h, LB_RT_EINVAL, "ptr_kind must be LB_RT_HOST or LB_RT_DEVICE");
  cudaMemcpyKind k = ptr_kind == LB_RT_HOST ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToDevice;
  CK(h, cudaMemcpyAsync(dst, src, bytes, k, h->stream));
  if (ptr_kind == LB_RT_HOST) CK(h, cudaStreamSynchronize(h->stream));
  return LB_RT_OK;
}

lb_rt_status reset_budget(lb_rt* h) {
  CK(h, cudaMemsetAsync(h->acc, 0, 8 * sizeof(double), h->stream));
  cudaError_t e = launch_total_energy(h->grid, h->Ni, h->pop[h->cur], h->ef[h->cur],
                                      h->cfg.storage, h->table, h->partials, h->partials_cap,
                                      h->acc, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "total energy");
  CK(h, cudaMemcpyAsync(h->acc + 1, h->acc, sizeof(double), cudaMemcpyDeviceToDevice, h->stream));
  return LB_RT_OK;
}

// nsteps steps; the last one also writes E, F of the new state to mE / mF
// (FP32 static step only; the caller checks that the epilogue form applies)
lb_rt_status run_steps(lb_rt* h, int nsteps, float* mE, float* mF) {
  if (h->timing) CK(h, cudaEventRecord(h->ev0, h->stream));
  int launches = 0;
  for (int s = 0; s < nsteps; ++s) {
    StepLaunch L{};
    L.g = h->grid;
    L.N = h->Ni;
    L.dpt = h->dpt;
    L.zc = h->zc;
    L.nzc = h->nzc;
    L.ctas = h->ctas;
    L.dt = (float)h->dt;
    L.collision = h->cfg.collision;
    L.lambda_iters = h->cfg.lambda_iters;
    L.in = h->pop[h->cur];
    L.out = h->pop[h->cur ^ 1];
    L.tmap_in = h->tmap_ok ? &h->tmap[h->cur] : nullptr;
    L.tmap_e = h->ef[0] && h->tmap_ok ? &h->emap[h->cur] : nullptr;
    L.e_in = h->ef[h->cur];
    L.e_out = h->ef[h->cur ^ 1];
    L.err = h->err;
    L.sc = h->pipelined;
    L.budget_partials = nullptr;
    L.partials_cap = h->partials_cap;
    if (s == nsteps - 1) {
      L.mom_E = mE;
      L.mom_F = mF;
    }
    int nblocks = 0;
    if (h->cfg.budget) {
      L.budget_partials = h->partials;
      CK(h, cudaMemsetAsync(h->partials, 0, sizeof(double) * 2 * h->partials_cap, h->stream));
    }
    cudaError_t e = h->cfg.moving
                        ? launch_step_moving(L, h->mc, h->table, h->cfg.storage, h->stream, &nblocks)
                        : launch_step_static(L, h->sc, h->table, h->cfg.storage, h->stream, &nblocks);
    if (e != cudaSuccess) return cuda_fail(h, e, "step kernel");
    ++launches;
    if (h->nfrozen) {
      e = launch_frozen(h->grid, h->Ni, h->N, h->d_int_of_ext, h->nfrozen, h->frozen_cells,
                        h->frozen_vals, h->pop[h->cur ^ 1], h->ef[h->cur ^ 1], h->cfg.storage,
                        h->table, h->cfg.budget ? h->acc + 6 : nullptr, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "frozen kernel");
    }
    if (h->cfg.budget) {
      e = launch_budget_finalize(h->partials, nblocks, h->acc, h->stream);
      if (e != cudaSuccess) return cuda_fail(h, e, "budget kernel");
    }
    h->cur ^= 1;
    ++h->steps;
  }
  if (h->timing) CK(h, cudaEventRecord(h->ev1, h->stream));
  h->last_nlaunch = launches;
  return LB_RT_OK;
}

// device address the kernels may write for a host pointer: page-locked
// mapped memory gives one, anything else nullptr
float* mapped_device_ptr(float* p) {
  if (!p) return nullptr;
  void* d = nullptr;
  if (cudaHostGetDevicePointer(&d, p, 0) != cudaSuccess) {
    (void)cudaGetLastError();
    return nullptr;
  }
  return static_cast<float*>(d);
}


}  // namespace

size_t lbrt::handle_device_bytes(const lb_rt_config& cfg, std::string& err) {
  lb_rt tmp;
  tmp.cfg = cfg;
  if (!build_directions(cfg, tmp.n, tmp.w, err)) return 0;
  tmp.N = (int)tmp.w.size();
  tmp.grid.nx = cfg.nx;
  tmp.grid.ny = cfg.ny;
  tmp.grid.nz = cfg.nz;
  plan_directions(&tmp);
  if (!cfg.moving && !tmp.dpt) {
    err = "no tile plan fits this direction set";
    return 0;
  }
  const size_t PX = ((size_t)(cfg.nx + GL + 1) + 7) / 8 * 8, PY = cfg.ny + 2, PZ = cfg.nz + 2;
  const size_t sites = (size_t)cfg.nx * cfg.ny * cfg.nz;
  size_t b = 2 * PX * PY * PZ * (size_t)tmp.Ni * elem_bytes(cfg.storage);
  if (cfg.storage != LB_RT_F32) b += 2 * PX * PY * PZ * sizeof(float);
  const size_t step_blocks = (size_t)((cfg.nx + 31) / 32) * cfg.ny * cfg.nz;
  b += 2 * sizeof(double) * std::max<size_t>(4096, step_blocks);
  b += (cfg.moving ? 6 : 4) * sites * sizeof(float);  // coefficient fields
  b += 10 * sites * sizeof(float);                      // moments staging for host outputs
  return b + 64 * 1024;
}

// Message for lb_rt_last_error(NULL) from a failed call that has no handle.
void lbrt::set_unbound_error(const std::string& m) { g_create_msg = m; }

extern "C" {

const char* lb_rt_version(void) { return "lbrt 0.1 (sm_103a)"; }

// With a NULL handle: the reason the calling thread's last lb_rt_create failed.
const char* lb_rt_last_error(const lb_rt* h) { return h ? h->msg.c_str() : g_create_msg.c_str(); }

lb_rt_status lb_rt_create(const lb_rt_config* cfg, lb_rt** out) {
  if (!cfg || !out) return LB_RT_EINVAL;
  *out = nullptr;
  lb_rt* h = new (std::nothrow) lb_rt();
  if (!h) return LB_RT_ENOMEM;
  h->cfg = *cfg;
  h->cfg.dirs = nullptr;
  h->cfg.weights = nullptr;
  auto bad = [&](const char* m) {
    g_create_msg = m;
    lb_rt_destroy(h);
    return LB_RT_EINVAL;
  };
  if (cfg->dims != 2 && cfg->dims != 3) return bad("dims must be 2 or 3");
  if (cfg->nx < 1 || cfg->ny < 1 || cfg->nz < 1) return bad("grid sizes must be >= 1");
  if (cfg->dims == 2 && cfg->nz != 1) return bad("dims == 2 needs nz == 1");
  if (!(cfg->cfl > 0.0 && cfg->cfl <= 1.0)) return bad("cfl must be in (0, 1]");
  if (!(cfg->dx > 0.0)) return bad("dx must be > 0");
  for (int a = 0; a < 3; ++a)
    if (cfg->bc[a] != LB_RT_PERIODIC && cfg->bc[a] != LB_RT_VACUUM) return bad("bad bc");
  if (cfg->storage != LB_RT_F32 && cfg->storage != LB_RT_F16_DEV &&
      cfg->storage != LB_RT_BF16_DEV)
    return bad("bad storage");
  if (cfg->collision != LB_RT_IMPLICIT_EXACT && cfg->collision != LB_RT_EXPLICIT &&
      cfg->collision != LB_RT_LAMBDA_K)
    return bad("bad collision");
  if (cfg->collision == LB_RT_LAMBDA_K && cfg->lambda_iters < 1)
    return bad("lambda_iters must be >= 1");
  if (cfg->moving && cfg->collision != LB_RT_IMPLICIT_EXACT)
    return bad("moving fluid supports the exact implicit collision only");
  const long long sites = (long long)cfg->nx * cfg->ny * cfg->nz;
  if (sites >= (1LL << 31)) return bad("more than 2^31 - 1 sites");
  std::string err;
  if (!build_directions(*cfg, h->n, h->w, err)) return bad(err.c_str());
  h->N = (int)h->w.size();
  if (h->N > LB_RT_MAX_DIRS) return bad("too many directions");
  if (cfg->dims == 2)
    for (int i = 0; i < h->N; ++i)
      if (h->n[3 * i + 2] != 0.0) return bad("2D grids need directions with n_z == 0");
  {
    std::string iso_err;
    h->iso = isotropic_table(h->n, h->w, cfg->dims, iso_err);
    if (cfg->collision != LB_RT_EXPLICIT && !h->iso) return bad(iso_err.c_str());
  }
  h->grid.nx = cfg->nx;
  h->grid.ny = cfg->ny;
  h->grid.nz = cfg->nz;
  h->grid.dims = cfg->dims;
  h->grid.sites = sites;
  for (int a = 0; a < 3; ++a) h->grid.periodic[a] = cfg->bc[a] == LB_RT_PERIODIC;
  // padded layout (see lb_rt_internal.h): rows of a multiple of 8 elements
  h->grid.PX = ((cfg->nx + GL + 1) + 7) / 8 * 8;
  h->grid.PY = cfg->ny + 2;
  h->grid.PZ = cfg->nz + 2;
  plan_directions(h);
  if (!h->cfg.moving && !h->dpt) return bad("no tile plan fits this direction set");
  h->grid.si = h->grid.PX;
  h->grid.sy = (long long)h->Ni * h->grid.PX;
  h->grid.sz = h->grid.sy * h->grid.PY;
  h->grid.total = h->grid.sz * h->grid.PZ;
  h->dt = cfg->cfl * cfg->dx;
  fill_table(h);

  cudaError_t e = cudaGetDevice(&h->device);
  if (e != cudaSuccess) {
    g_create_msg = std::string("cudaGetDevice: ") + cudaGetErrorString(e);
    lb_rt_destroy(h);
    return LB_RT_ECUDA;
  }
  if (cfg->stream) {
    h->stream = (cudaStream_t)cfg->stream;
  } else {
    e = cudaStreamCreateWithFlags(&h->stream, cudaStreamNonBlocking);
    h->own_stream = (e == cudaSuccess);
  }
  h->pop_bytes = (size_t)h->grid.total * elem_bytes(cfg->storage);
  const int max_blocks = 4096;
  auto alloc = [&](void** p, size_t b) {
    if (e != cudaSuccess) return;
    e = cudaMalloc(p, b);
  };
  alloc(&h->pop[0], h->pop_bytes);
  alloc(&h->pop[1], h->pop_bytes);
  if (cfg->storage != LB_RT_F32) {
    h->ef_bytes = sizeof(float) * (size_t)h->grid.PX * h->grid.PY * h->grid.PZ;
    alloc((void**)&h->ef[0], h->ef_bytes);
    alloc((void**)&h->ef[1], h->ef_bytes);
  }
  // budget partials: one slot pair per CTA of the step kernel; every step
  // kernel's grid is at most ceil(nx/32) x ny x nz CTAs
  const long long step_blocks = (long long)((cfg->nx + 31) / 32) * cfg->ny * cfg->nz;
  h->partials_cap = (int)std::max<long long>(max_blocks, step_blocks);
  alloc((void**)&h->partials, sizeof(double) * 2 * h->partials_cap);
  alloc((void**)&h->acc, sizeof(double) * 8);
  alloc((void**)&h->d_int_of_ext, sizeof(int) * h->N);
  alloc((void**)&h->err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaHostAlloc((void**)&h->err_host, sizeof(unsigned), cudaHostAllocDefault);
  if (e != cudaSuccess) {
    g_create_msg = std::string("allocation: ") + cudaGetErrorString(e);
    lb_rt_destroy(h);
    return e == cudaErrorMemoryAllocation ? LB_RT_ENOMEM : LB_RT_ECUDA;
  }
  h->sc = StaticCoef{nullptr, nullptr, nullptr, nullptr, 0.f, 0.f, 0.f, 0.f};
  h->mc = MovingCoef{nullptr, nullptr, nullptr, nullptr, 0.f, 0.f, 0.f};
  // zero both buffers: ghost cells of vacuum faces stay zero for good
  e = cudaMemsetAsync(h->pop[0], 0, h->pop_bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->pop[1], 0, h->pop_bytes, h->stream);
  for (int b = 0; b < 2; ++b)
    if (e == cudaSuccess && h->ef[b]) e = cudaMemsetAsync(h->ef[b], 0, h->ef_bytes, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->acc, 0, sizeof(double) * 8, h->stream);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(h->d_int_of_ext, h->int_of_ext.data(), sizeof(int) * h->N,
                        cudaMemcpyHostToDevice, h->stream);
  if (e == cudaSuccess) e = cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(h->stream);
  if (e != cudaSuccess) {
    g_create_msg = std::string("init: ") + cudaGetErrorString(e);
    lb_rt_destroy(h);
    return LB_RT_ECUDA;
  }
  const bool tiled = !cfg->moving || h->dpt > 0;
  if (tiled) {
    std::string terr;
    for (int b = 0; b < 2; ++b) {
      const bool ok =
          cfg->storage == LB_RT_F32
              ? make_pop_tensor_map(&h->tmap[b], h->grid, h->Ni, h->pop[b], h->dpt, h->zc, terr)
              : make_pop16_tensor_map(&h->tmap[b], h->grid, h->Ni, h->pop[b], cfg->storage,
                                      h->dpt, h->zc, terr) &&
                    make_e_tensor_map(&h->emap[b], h->grid, h->ef[b], h->zc, terr);
      if (!ok) {
        g_create_msg = terr;
        lb_rt_destroy(h);
        return LB_RT_ECUDA;
      }
    }
    h->tmap_ok = true;
    e = plan_static_grid(h->grid, h->Ni, h->dpt, h->zc, cfg->storage, &h->nzc, &h->ctas,
                         cfg->moving != 0, h->pipelined);
    if (e != cudaSuccess && h->pipelined) {
      // the pipelined kernel cannot be resident with this plan on this
      // device: the first-generation kernel runs the same plan
      (void)cudaGetLastError();
      h->pipelined = false;
      e = plan_static_grid(h->grid, h->Ni, h->dpt, h->zc, cfg->storage, &h->nzc, &h->ctas,
                           cfg->moving != 0, false);
    }
    if (e != cudaSuccess) {
      g_create_msg = std::string("static kernel grid: ") + cudaGetErrorString(e);
      lb_rt_destroy(h);
      return LB_RT_ECUDA;
    }
  }
  *out = h;
  return LB_RT_OK;
}

void lb_rt_destroy(lb_rt* h) {
  if (!h) return;
  if (h->stream) cudaStreamSynchronize(h->stream);
  for (void* p : h->pop) cudaFree(p);
  for (void* p : h->ef) cudaFree(p);
  for (void* p : h->fld) cudaFree(p);
  cudaFree(h->frozen_cells);
  cudaFree(h->frozen_vals);
  cudaFree(h->partials);
  cudaFree(h->acc);
  cudaFree(h->d_int_of_ext);
  cudaFree(h->err);
  if (h->err_host) cudaFreeHost(h->err_host);
  cudaFree(h->scratch);
  if (h->ev0) cudaEventDestroy(h->ev0);
  if (h->ev1) cudaEventDestroy(h->ev1);
  if (h->own_stream) cudaStreamDestroy(h->stream);
  delete h;
}

lb_rt_status lb_rt_set_fluid(lb_rt* h, const lb_rt_fluid* f, int ptr_kind) {
  if (!h) return LB_RT_EINVAL;
  if (!f) return fail(h, LB_RT_EINVAL, "null fluid");
  if (ptr_kind != LB_RT_HOST && ptr_kind != LB_RT_DEVICE && ptr_kind != LB_RT_HOST_MAPPED)
    return fail(h, LB_RT_EINVAL, "bad ptr_kind");
  const size_t sb = sizeof(float) * h->grid.sites;
  auto put = [&](int slot, const float* src, size_t bytes, const float** dst) -> lb_rt_status {
    if (!src) {
      *dst = nullptr;
      return LB_RT_OK;
    }
    if (ptr_kind == LB_RT_HOST_MAPPED) {
      const float* d = mapped_device_ptr(const_cast<float*>(src));
      if (!d) return fail(h, LB_RT_EINVAL, "LB_RT_HOST_MAPPED field is not page-locked mapped memory");
      *dst = d;
      return LB_RT_OK;
    }
    if (!h->fld[slot]) CK(h, cudaMalloc((void**)&h->fld[slot], bytes));
    lb_rt_status st = copy_in(h, h->fld[slot], src, bytes, ptr_kind);
    *dst = h->fld[slot];
    return st;
  };
  lb_rt_status st = LB_RT_OK;
  if (!h->cfg.moving) {
    if (f->v || f->kt_a || f->kt_0 || f->eta_t)
      return fail(h, LB_RT_EINVAL, "moving-fluid fields given to a static handle");
    StaticCoef c{};
    if ((st = put(0, f->kappa_a, sb, &c.ka)) != LB_RT_OK) return st;
    if ((st = put(1, f->kappa_0, sb, &c.k0)) != LB_RT_OK) return st;
    if ((st = put(2, f->lambda, sb, &c.lam)) != LB_RT_OK) return st;
    if ((st = put(3, f->eta, sb, &c.eta)) != LB_RT_OK) return st;
    c.ka_s = f->kappa_a_s;
    c.k0_s = f->kappa_0_s;
    c.lam_s = f->lambda_s;
    c.eta_s = f->eta_s;
    h->sc = c;
  } else {
    if (f->kappa_a || f->kappa_0 || f->lambda || f->eta)
      return fail(h, LB_RT_EINVAL, "static-fluid fields given to a moving handle");
    MovingCoef c{};
    if ((st = put(4, f->v, 3 * sb, &c.v)) != LB_RT_OK) return st;
    if ((st = put(5, f->kt_a, sb, &c.kta)) != LB_RT_OK) return st;
    if ((st = put(6, f->kt_0, sb, &c.kt0)) != LB_RT_OK) return st;
    if ((st = put(7, f->eta_t, sb, &c.etat)) != LB_RT_OK) return st;
    c.kta_s = f->kt_a_s;
    c.kt0_s = f->kt_0_s;
    c.etat_s = f->eta_t_s;
    h->mc = c;
  }
  return LB_RT_OK;
}

lb_rt_status lb_rt_set_state(lb_rt* h, const float* data, int kind, int ptr_kind) {
  if (!h) return LB_RT_EINVAL;
  if (!data) return fail(h, LB_RT_EINVAL, "null data");
  size_t count;
  if (kind == LB_RT_STATE_POPULATIONS) count = (size_t)h->grid.sites * h->N;
  else if (kind == LB_RT_STATE_ISOTROPIC) count = (size_t)h->grid.sites;
  else if (kind == LB_RT_STATE_P1) count = 4 * (size_t)h->grid.sites;
  else return fail(h, LB_RT_EINVAL, "bad state kind");
  const float* src = data;
  float* tmp = nullptr;
  if (ptr_kind == LB_RT_HOST) {
    CK(h, cudaMalloc((void**)&tmp, count * sizeof(float)));
    cudaError_t e = cudaMemcpyAsync(tmp, data, count * sizeof(float), cudaMemcpyHostToDevice,
                                    h->stream);
    if (e != cudaSuccess) {
      cudaFree(tmp);
      return cuda_fail(h, e, "set_state copy");
    }
    src = tmp;
  } else if (ptr_kind != LB_RT_DEVICE) {
    return fail(h, LB_RT_EINVAL, "bad ptr_kind");
  }
  h->cur = 0;
  cudaError_t e = launch_init_state(h->grid, h->Ni, h->N, h->d_int_of_ext, src, kind, h->pop[0],
                                    h->ef[0], h->cfg.storage, h->table, h->stream);
  if (tmp) {
    cudaError_t e2 = cudaStreamSynchronize(h->stream);
    cudaFree(tmp);
    if (e == cudaSuccess) e = e2;
  }
  if (e != cudaSuccess) return cuda_fail(h, e, "set_state");
  h->steps = 0;
  return reset_budget(h);
}

lb_rt_status lb_rt_set_frozen(lb_rt* h, const int64_t* cells, int ncells, const float* values) {
  if (!h) return LB_RT_EINVAL;
  if (ncells < 0) return fail(h, LB_RT_EINVAL, "ncells < 0");
  CK(h, cudaStreamSynchronize(h->stream));
  cudaFree(h->frozen_cells);
  cudaFree(h->frozen_vals);
  h->frozen_cells = nullptr;
  h->frozen_vals = nullptr;
  h->nfrozen = 0;
  if (ncells == 0) return LB_RT_OK;
  if (!cells || !values) return fail(h, LB_RT_EINVAL, "null frozen arrays");
  for (int k = 0; k < ncells; ++k)
    if (cells[k] < 0 || cells[k] >= h->grid.sites)
      return fail(h, LB_RT_EINVAL, "frozen cell index out of range");
  CK(h, cudaMalloc((void**)&h->frozen_cells, sizeof(int64_t) * ncells));
  CK(h, cudaMalloc((void**)&h->frozen_vals, sizeof(float) * ncells * (size_t)h->N));
  CK(h, cudaMemcpy(h->frozen_cells, cells, sizeof(int64_t) * ncells, cudaMemcpyHostToDevice));
  CK(h, cudaMemcpy(h->frozen_vals, values, sizeof(float) * ncells * (size_t)h->N,
                   cudaMemcpyHostToDevice));
  h->nfrozen = ncells;
  return LB_RT_OK;
}


lb_rt_status lb_rt_step(lb_rt* h, int nsteps) {
  if (!h) return LB_RT_EINVAL;
  if (nsteps < 0) return fail(h, LB_RT_EINVAL, "nsteps < 0");
  return run_steps(h, nsteps, nullptr, nullptr);
}

lb_rt_status lb_rt_step_moments(lb_rt* h, int nsteps, float* E, float* F, int ptr_kind) {
  if (!h) return LB_RT_EINVAL;
  if (nsteps < 0) return fail(h, LB_RT_EINVAL, "nsteps < 0");
  if (ptr_kind != LB_RT_HOST && ptr_kind != LB_RT_DEVICE)
    return fail(h, LB_RT_EINVAL, "bad ptr_kind");
  const bool epilogue = nsteps > 0 && (E || F) && !h->cfg.moving &&
                        h->cfg.storage == LB_RT_F32 && h->nfrozen == 0 && h->iso;
  if (!epilogue) {
    const lb_rt_status st = run_steps(h, nsteps, nullptr, nullptr);
    if (st != LB_RT_OK) return st;
    return lb_rt_moments(h, E, F, nullptr, nullptr, ptr_kind);
  }
  const long long S = h->grid.sites;
  float *dE = E, *dF = F;
  bool stageE = false, stageF = false;
  if (ptr_kind == LB_RT_HOST) {
    dE = mapped_device_ptr(E);
    dF = mapped_device_ptr(F);
    stageE = E && !dE;
    stageF = F && !dF;
    if ((stageE || stageF) && !h->scratch)
      CK(h, cudaMalloc((void**)&h->scratch, sizeof(float) * 10 * S));
    if (stageE) dE = h->scratch;
    if (stageF) dF = h->scratch + S;
  }
  const lb_rt_status st = run_steps(h, nsteps, dE, dF);
  if (st != LB_RT_OK) return st;
  if (stageE) CK(h, cudaMemcpyAsync(E, dE, sizeof(float) * S, cudaMemcpyDeviceToHost, h->stream));
  if (stageF)
    CK(h, cudaMemcpyAsync(F, dF, sizeof(float) * 3 * S, cudaMemcpyDeviceToHost, h->stream));
  if (ptr_kind == LB_RT_HOST) return lb_rt_sync(h);
  return LB_RT_OK;
}

lb_rt_status lb_rt_sync(lb_rt* h) {
  if (!h) return LB_RT_EINVAL;
  // the error word comes back with the same synchronisation
  CK(h, cudaMemcpyAsync(h->err_host, h->err, sizeof(unsigned), cudaMemcpyDeviceToHost, h->stream));
  CK(h, cudaStreamSynchronize(h->stream));
  const unsigned word = *h->err_host;
  if (word) {
    // reported once: the word is cleared so that a restored or re-set state
    // can be stepped again (the state itself is not trusted, see lb_rt.h)
    *h->err_host = 0;
    CK(h, cudaMemsetAsync(h->err, 0, sizeof(unsigned), h->stream));
    char buf[96];
    std::snprintf(buf, sizeof buf, "device error word 0x%08x", word);
    return fail(h, LB_RT_ETIMEDOUT, buf);
  }
  return LB_RT_OK;
}

lb_rt_status lb_rt_moments(lb_rt* h, float* E, float* F, float* P, lb_rt_budget* budget,
                           int ptr_kind) {
  if (!h) return LB_RT_EINVAL;
  if (ptr_kind != LB_RT_HOST && ptr_kind != LB_RT_DEVICE)
    return fail(h, LB_RT_EINVAL, "bad ptr_kind");
  const long long S = h->grid.sites;
  if (E || F || P) {
    float *dE = E, *dF = F, *dP = P;
    if (ptr_kind == LB_RT_HOST) {
      if (!h->scratch) CK(h, cudaMalloc((void**)&h->scratch, sizeof(float) * 10 * S));
      dE = E ? h->scratch : nullptr;
      dF = F ? h->scratch + S : nullptr;
      dP = P ? h->scratch + 4 * S : nullptr;
    }
    cudaError_t e = launch_moments(h->grid, h->Ni, h->pop[h->cur], h->ef[h->cur],
                                   h->cfg.storage, h->table, dE, dF, dP, h->stream);
    if (e != cudaSuccess) return cuda_fail(h, e, "moments kernel");
    if (ptr_kind == LB_RT_HOST) {
      if (E) CK(h, cudaMemcpyAsync(E, dE, sizeof(float) * S, cudaMemcpyDeviceToHost, h->stream));
      if (F) CK(h, cudaMemcpyAsync(F, dF, sizeof(float) * 3 * S, cudaMemcpyDeviceToHost, h->stream));
      if (P) CK(h, cudaMemcpyAsync(P, dP, sizeof(float) * 6 * S, cudaMemcpyDeviceToHost, h->stream));
    }
  }
  if (budget) {
    double a[8];
    CK(h, cudaMemcpyAsync(a, h->acc, sizeof(a), cudaMemcpyDeviceToHost, h->stream));
    CK(h, cudaStreamSynchronize(h->stream));
    budget->total = a[0];
    budget->initial = a[1];
    budget->outflow = a[2];
    budget->source = a[3];
    budget->injection = a[4];
    budget->steps = (long long)a[5];
  }
  if (ptr_kind == LB_RT_HOST) return lb_rt_sync(h);
  return LB_RT_OK;
}

lb_rt_status lb_rt_coupling(lb_rt* h, float* J, float* H, float* S, int ptr_kind) {
  if (!h) return LB_RT_EINVAL;
  if (ptr_kind != LB_RT_HOST && ptr_kind != LB_RT_DEVICE)
    return fail(h, LB_RT_EINVAL, "bad ptr_kind");
  if (!J && !H && !S) return LB_RT_OK;
  const long long S_ = h->grid.sites;
  // a static fluid is the moving one at rest with its own opacities
  MovingCoef c = h->mc;
  if (!h->cfg.moving) {
    c = MovingCoef{nullptr, h->sc.ka, h->sc.k0, h->sc.eta, h->sc.ka_s, h->sc.k0_s, h->sc.eta_s};
  }
  float *dJ = J, *dH = H, *dS = S;
  if (ptr_kind == LB_RT_HOST) {
    if (!h->scratch) CK(h, cudaMalloc((void**)&h->scratch, sizeof(float) * 10 * S_));
    dJ = J ? h->scratch : nullptr;
    dH = H ? h->scratch + S_ : nullptr;
    dS = S ? h->scratch + 4 * S_ : nullptr;
  }
  cudaError_t e = launch_coupling(h->grid, h->Ni, h->pop[h->cur], h->ef[h->cur], h->cfg.storage,
                                  h->table, c, dJ, dH, dS, h->stream);
  if (e != cudaSuccess) return cuda_fail(h, e, "coupling kernel");
  if (ptr_kind == LB_RT_HOST) {
    if (J) CK(h, cudaMemcpyAsync(J, dJ, sizeof(float) * S_, cudaMemcpyDeviceToHost, h->stream));
    if (H) CK(h, cudaMemcpyAsync(H, dH, sizeof(float) * 3 * S_, cudaMemcpyDeviceToHost, h->stream));
    if (S) CK(h, cudaMemcpyAsync(S, dS, sizeof(float) * 4 * S_, cudaMemcpyDeviceToHost, h->stream));
    return lb_rt_sync(h);
  }
  return LB_RT_OK;
}

lb_rt_status lb_rt_get_populations(lb_rt* h, float* out, int ptr_kind) {
  if (!h || !out) return fail(h, LB_RT_EINVAL, "null argument");
  const size_t count = (size_t)h->grid.sites * h->N;
  float* dst = out;
  float* tmp = nullptr;
  if (ptr_kind == LB_RT_HOST) {
    CK(h, cudaMalloc((void**)&tmp, count * sizeof(float)));
    dst = tmp;
  } else if (ptr_kind != LB_RT_DEVICE) {
    return fail(h, LB_RT_EINVAL, "bad ptr_kind");
  }
  cudaError_t e =
      launch_decode(h->grid, h->N, h->d_int_of_ext, h->pop[h->cur], h->ef[h->cur], h->cfg.storage,
                    h->table, dst, h->stream);
  if (e == cudaSuccess && tmp)
    e = cudaMemcpyAsync(out, tmp, count * sizeof(float), cudaMemcpyDeviceToHost, h->stream);
  if (e == cudaSuccess && tmp) e = cudaStreamSynchronize(h->stream);
  cudaFree(tmp);
  if (e != cudaSuccess) return cuda_fail(h, e, "get_populations");
  return ptr_kind == LB_RT_HOST ? lb_rt_sync(h) : LB_RT_OK;
}

size_t lb_rt_state_bytes(const lb_rt* h) {
  if (!h) return 0;
  size_t b = 64 + h->pop_bytes + 8 * sizeof(double);
  if (h->ef[0]) b += h->ef_bytes;
  return b;
}

lb_rt_status lb_rt_save_state(lb_rt* h, void* buf, size_t bytes) {
  if (!h || !buf) return fail(h, LB_RT_EINVAL, "null argument");
  if (bytes < lb_rt_state_bytes(h)) return fail(h, LB_RT_EINVAL, "buffer too small");
  char* p = static_cast<char*>(buf);
  long long hdr[8] = {0x4c42525453544154LL, h->N, h->grid.sites, h->cfg.storage, h->steps, 0, 0, 0};
  std::memcpy(p, hdr, 64);
  p += 64;
  CK(h, cudaMemcpyAsync(p, h->pop[h->cur], h->pop_bytes, cudaMemcpyDeviceToHost, h->stream));
  p += h->pop_bytes;
  if (h->ef[0]) {
    CK(h, cudaMemcpyAsync(p, h->ef[h->cur], h->ef_bytes, cudaMemcpyDeviceToHost, h->stream));
    p += h->ef_bytes;
  }
  CK(h, cudaMemcpyAsync(p, h->acc, 8 * sizeof(double), cudaMemcpyDeviceToHost, h->stream));
  return lb_rt_sync(h);
}

lb_rt_status lb_rt_restore_state(lb_rt* h, const void* buf, size_t bytes) {
  if (!h || !buf) return fail(h, LB_RT_EINVAL, "null argument");
  if (bytes < lb_rt_state_bytes(h)) return fail(h, LB_RT_EINVAL, "buffer too small");
  const char* p = static_cast<const char*>(buf);
  long long hdr[8];
  std::memcpy(hdr, p, 64);
  if (hdr[0] != 0x4c42525453544154LL || hdr[1] != h->N || hdr[2] != h->grid.sites ||
      hdr[3] != h->cfg.storage)
    return fail(h, LB_RT_EINVAL, "state does not match this handle");
  p += 64;
  CK(h, cudaStreamSynchronize(h->stream));
  CK(h, cudaMemcpy(h->pop[h->cur], p, h->pop_bytes, cudaMemcpyHostToDevice));
  p += h->pop_bytes;
  if (h->ef[0]) {
    CK(h, cudaMemcpy(h->ef[h->cur], p, h->ef_bytes, cudaMemcpyHostToDevice));
    p += h->ef_bytes;
  }
  CK(h, cudaMemcpy(h->acc, p, 8 * sizeof(double), cudaMemcpyHostToDevice));
  h->steps = hdr[4];
  return LB_RT_OK;
}

lb_rt_status lb_rt_directions(const lb_rt* h, int* ndir, double* dirs, double* weights,
                              int8_t* signs) {
  if (!h) return LB_RT_EINVAL;
  if (ndir) *ndir = h->N;
  for (int i = 0; i < h->N; ++i) {
    for (int a = 0; a < 3; ++a) {
      if (dirs) dirs[3 * i + a] = h->n[3 * i + a];
      if (signs) signs[3 * i + a] = h->n[3 * i + a] < 0.0 ? -1 : 1;
    }
    if (weights) weights[i] = h->w[i];
  }
  return LB_RT_OK;
}

lb_rt_status lb_rt_enable_timing(lb_rt* h, int on) {
  if (!h) return LB_RT_EINVAL;
  if (on && !h->ev0) {
    CK(h, cudaEventCreate(&h->ev0));
    CK(h, cudaEventCreate(&h->ev1));
  }
  h->timing = on != 0;
  return LB_RT_OK;
}

lb_rt_status lb_rt_last_step_ms(lb_rt* h, float* ms, int* nlaunch) {
  if (!h) return LB_RT_EINVAL;
  if (!h->timing) return fail(h, LB_RT_EINVAL, "timing not enabled");
  CK(h, cudaEventSynchronize(h->ev1));
  float t = 0.f;
  CK(h, cudaEventElapsedTime(&t, h->ev0, h->ev1));
  if (ms) *ms = t;
  if (nlaunch) *nlaunch = h->last_nlaunch;
  return LB_RT_OK;
}

}  // extern "C"
