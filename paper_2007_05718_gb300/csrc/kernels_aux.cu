// Auxiliary kernels on the padded population layout: initial populations,
// moments (Eqs. moments_discrete, higher_moments), decoding to dense
// float32, frozen-cell overwrite and the FP64 energy-budget reductions.
// Every population write also writes the site's periodic ghost mirrors.
#include <algorithm>

#include "lb_rt_internal.h"

namespace lbrt {

namespace {

constexpr int BLK = 256;

__device__ __forceinline__ void site_xyz(const Grid& g, long long s, int& x, int& y, int& z) {
  x = (int)(s % g.nx);
  const long long r = s / g.nx;
  y = (int)(r % g.ny);
  z = (int)(r / g.ny);
}

__device__ __forceinline__ float load_pop(const void* pop, const Grid& g, int i, int z, int y,
                                          int x) {
  return static_cast<const float*>(pop)[pidx(g, i, z, y, x)];
}

// kind: populations (data [Next][sites] in the external order), isotropic
// (I_i = w_i E0) or P1 (I_i = w_i (E0 + d n_i.F0)).  Inert padding directions
// (w = 0, n = 0) get 0.
__global__ void k_init_state(Grid g, int Ni, int Next, const int* __restrict__ int_of_ext,
                             const float* __restrict__ data, int kind, float* __restrict__ pop,
                             DirTable t) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.sites) return;
  int x, y, z;
  site_xyz(g, s, x, y, z);
  const float d = (float)g.dims;
  if (kind == LB_RT_STATE_POPULATIONS) {
    for (int e = 0; e < Next; ++e)
      store_pop(pop, g, int_of_ext[e], z, y, x, data[(size_t)e * g.sites + s]);
    return;
  }
  for (int i = 0; i < Ni; ++i) {
    const float4 nw = t.nw[i];
    float v;
    if (kind == LB_RT_STATE_ISOTROPIC) {
      v = nw.w * data[s];
    } else {
      v = nw.w * (data[s] + d * (nw.x * data[g.sites + s] + nw.y * data[2 * g.sites + s] +
                                 nw.z * data[3 * g.sites + s]));
    }
    store_pop(pop, g, i, z, y, x, v);
  }
}

// E, F, P per site: sums over directions in the table order.
__global__ void k_moments(Grid g, int N, const void* __restrict__ pop, float* __restrict__ E,
                          float* __restrict__ F, float* __restrict__ P, DirTable t) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.sites) return;
  int x, y, z;
  site_xyz(g, s, x, y, z);
  float e = 0, fx = 0, fy = 0, fz = 0, pxx = 0, pxy = 0, pxz = 0, pyy = 0, pyz = 0, pzz = 0;
  for (int i = 0; i < N; ++i) {
    const float v = load_pop(pop, g, i, z, y, x);
    const float4 nw = t.nw[i];
    e += v;
    fx = fmaf(nw.x, v, fx);
    fy = fmaf(nw.y, v, fy);
    fz = fmaf(nw.z, v, fz);
    pxx = fmaf(nw.x * nw.x, v, pxx);
    pxy = fmaf(nw.x * nw.y, v, pxy);
    pxz = fmaf(nw.x * nw.z, v, pxz);
    pyy = fmaf(nw.y * nw.y, v, pyy);
    pyz = fmaf(nw.y * nw.z, v, pyz);
    pzz = fmaf(nw.z * nw.z, v, pzz);
  }
  if (E) E[s] = e;
  if (F) {
    F[s] = fx;
    F[g.sites + s] = fy;
    F[2 * g.sites + s] = fz;
  }
  if (P) {
    P[s] = pxx;
    P[g.sites + s] = pxy;
    P[2 * g.sites + s] = pxz;
    P[3 * g.sites + s] = pyy;
    P[4 * g.sites + s] = pyz;
    P[5 * g.sites + s] = pzz;
  }
}

// Dense [Next][sites] float32 copy in the external direction order.
__global__ void k_decode(Grid g, int Next, const int* __restrict__ int_of_ext,
                         const void* __restrict__ pop, float* __restrict__ out) {
  const long long total = g.sites * (long long)Next;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int e = (int)(k / g.sites);
    int x, y, z;
    site_xyz(g, k % g.sites, x, y, z);
    out[k] = load_pop(pop, g, int_of_ext[e], z, y, x);
  }
}

// Frozen cells: overwrite, and add (prescribed - collided) energy to the
// FP64 injection accumulator.
__global__ void k_frozen(Grid g, int Next, const int* __restrict__ int_of_ext, int ncells,
                         const int64_t* __restrict__ cells, const float* __restrict__ vals,
                         float* __restrict__ pop, double* injection) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  int x, y, z;
  site_xyz(g, cells[c], x, y, z);
  double add = 0.0;
  for (int e = 0; e < Next; ++e) {
    const int i = int_of_ext[e];
    const float v = vals[(size_t)c * Next + e];
    add += (double)v - (double)pop[pidx(g, i, z, y, x)];
    store_pop(pop, g, i, z, y, x, v);
  }
  if (injection) atomicAdd(injection, add);
}

// acc layout: [0] total, [1] initial, [2] outflow, [3] source, [4] injection,
// [5] steps, [6] injection of the current step (added by the frozen kernel).
// partials: [nblocks][2] = (sum E*, sum E_collided) of the step just taken.
__global__ void k_budget_finalize(const double* __restrict__ partials, int nblocks, double* acc) {
  __shared__ double sa[BLK], sb[BLK];
  double a = 0.0, b = 0.0;
  for (int k = threadIdx.x; k < nblocks; k += blockDim.x) {
    a += partials[2 * k];
    b += partials[2 * k + 1];
  }
  sa[threadIdx.x] = a;
  sb[threadIdx.x] = b;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) {
      sa[threadIdx.x] += sa[threadIdx.x + w];
      sb[threadIdx.x] += sb[threadIdx.x + w];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double estar = sa[0], ecoll = sb[0];
    const double inj = acc[6];
    acc[2] += acc[0] - estar;   // outflow through vacuum faces
    acc[3] += ecoll - estar;    // collision source
    acc[4] += inj;
    acc[0] = ecoll + inj;
    acc[5] += 1.0;
    acc[6] = 0.0;
  }
}

// sum over sites of sum_i I_i in FP64: per-block partials, then one block.
__global__ void k_total_partials(Grid g, int N, const void* __restrict__ pop,
                                 double* __restrict__ partials) {
  __shared__ double sh[BLK];
  double acc = 0.0;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < g.sites;
       s += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    site_xyz(g, s, x, y, z);
    float e = 0.f;
    for (int i = 0; i < N; ++i) e += load_pop(pop, g, i, z, y, x);
    acc += (double)e;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

__global__ void k_sum_partials(const double* __restrict__ partials, int n, double* out) {
  __shared__ double sh[BLK];
  double a = 0.0;
  for (int k = threadIdx.x; k < n; k += blockDim.x) a += partials[k];
  sh[threadIdx.x] = a;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) *out = sh[0];
}

unsigned grid1d(long long n) { return (unsigned)((n + BLK - 1) / BLK); }

}  // namespace

cudaError_t launch_init_state(const Grid& g, int Ni, int Next, const int* int_of_ext,
                              const float* data, int kind, void* pop, int storage,
                              const DirTable& t, cudaStream_t s) {
  if (storage != ST_F32) return cudaErrorNotSupported;
  k_init_state<<<grid1d(g.sites), BLK, 0, s>>>(g, Ni, Next, int_of_ext, data, kind,
                                               static_cast<float*>(pop), t);
  return cudaGetLastError();
}

cudaError_t launch_moments(const Grid& g, int N, const void* pop, int storage, const DirTable& t,
                           float* E, float* F, float* P, cudaStream_t s) {
  if (storage != ST_F32) return cudaErrorNotSupported;
  k_moments<<<grid1d(g.sites), BLK, 0, s>>>(g, N, pop, E, F, P, t);
  return cudaGetLastError();
}

cudaError_t launch_decode(const Grid& g, int Next, const int* int_of_ext, const void* pop,
                          int storage, float* out, cudaStream_t s) {
  if (storage != ST_F32) return cudaErrorNotSupported;
  k_decode<<<1024, BLK, 0, s>>>(g, Next, int_of_ext, pop, out);
  return cudaGetLastError();
}

cudaError_t launch_frozen(const Grid& g, int Next, const int* int_of_ext, int ncells,
                          const int64_t* cells, const float* vals, void* pop, int storage,
                          double* injection_acc, cudaStream_t s) {
  if (storage != ST_F32) return cudaErrorNotSupported;
  if (ncells <= 0) return cudaSuccess;
  k_frozen<<<(ncells + BLK - 1) / BLK, BLK, 0, s>>>(g, Next, int_of_ext, ncells, cells, vals,
                                                    static_cast<float*>(pop), injection_acc);
  return cudaGetLastError();
}

cudaError_t launch_budget_finalize(const double* partials, int nblocks, double* acc,
                                   cudaStream_t s) {
  k_budget_finalize<<<1, BLK, 0, s>>>(partials, nblocks, acc);
  return cudaGetLastError();
}

cudaError_t launch_total_energy(const Grid& g, int N, const void* pop, int storage,
                                double* partials, int max_blocks, double* out, cudaStream_t s) {
  if (storage != ST_F32) return cudaErrorNotSupported;
  int nb = (int)std::min<long long>((long long)max_blocks, (long long)grid1d(g.sites));
  if (nb < 1) nb = 1;
  k_total_partials<<<nb, BLK, 0, s>>>(g, N, pop, partials);
  k_sum_partials<<<1, BLK, 0, s>>>(partials, nb, out);
  return cudaGetLastError();
}

}  // namespace lbrt
