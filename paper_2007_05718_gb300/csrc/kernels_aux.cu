// Auxiliary kernels on the padded population layout: initial populations,
// moments (Eqs. moments_discrete, higher_moments), decoding to dense
// float32, frozen-cell overwrite and the FP64 energy-budget reductions.
// Every population write also writes the site's periodic ghost mirrors.
#include <algorithm>
#include <type_traits>

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

// ---- 16-bit storage: f_i = I_i / w_i = E^ (1 + q_i), E^ = max(E, 1e-30) --

constexpr float EPS_E = 1e-30f;

__device__ __forceinline__ long long eidx(const Grid& g, int z, int y, int x) {
  return (long long)(z + 1) * g.PX * g.PY + (long long)(y + 1) * g.PX + x + GL;
}

template <class ST> __device__ __forceinline__ float to_f(ST v);
template <> __device__ __forceinline__ float to_f<__half>(__half v) { return __half2float(v); }
template <> __device__ __forceinline__ float to_f<__nv_bfloat16>(__nv_bfloat16 v) {
  return __bfloat162float(v);
}
template <class ST> __device__ __forceinline__ ST from_f(float v);
template <> __device__ __forceinline__ __half from_f<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// E^ of a site and every periodic mirror.
__device__ __forceinline__ void store_e_site(float* e, const Grid& g, int z, int y, int x, float v) {
  int xs[3], ys[3], zs[3];
  const int nxs = mirrors(x, g.nx, g.periodic[0], GL, xs);
  const int nys = mirrors(y, g.ny, g.periodic[1], 1, ys);
  const int nzs = mirrors(z, g.nz, g.periodic[2], 1, zs);
  for (int a = 0; a < nzs; ++a)
    for (int b = 0; b < nys; ++b)
      for (int c = 0; c < nxs; ++c)
        e[(long long)zs[a] * g.PX * g.PY + (long long)ys[b] * g.PX + xs[c]] = v;
}

// Encode f_i (per internal direction, from `kind` and `data` as in
// k_init_state) into q_i and E^.  Inert padding directions keep q = 0.
template <class ST>
__global__ void k_init_state16(Grid g, int Ni, int Next, const int* __restrict__ int_of_ext,
                               const float* __restrict__ data, int kind, ST* __restrict__ pop,
                               float* __restrict__ e, DirTable t) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.sites) return;
  int x, y, z;
  site_xyz(g, s, x, y, z);
  const float d = (float)g.dims;
  // f_i of internal direction i; E = sum_i w_i f_i
  auto f_of = [&](int i) -> float {
    const float4 nw = t.nw[i];
    if (kind == LB_RT_STATE_ISOTROPIC) return data[s];
    return data[s] + d * (nw.x * data[g.sites + s] + nw.y * data[2 * g.sites + s] +
                          nw.z * data[3 * g.sites + s]);
  };
  float E = 0.f;
  if (kind == LB_RT_STATE_POPULATIONS) {
    for (int ex = 0; ex < Next; ++ex) E += data[(size_t)ex * g.sites + s];
  } else if (kind == LB_RT_STATE_ISOTROPIC) {
    E = data[s];
  } else {
    for (int i = 0; i < Ni; ++i) E = fmaf(t.nw[i].w, f_of(i), E);
  }
  const float Eh = fmaxf(E, EPS_E);
  const float ri = 1.f / Eh;
  store_e_site(e, g, z, y, x, Eh);
  if (kind == LB_RT_STATE_POPULATIONS) {
    for (int ex = 0; ex < Next; ++ex) {
      const int i = int_of_ext[ex];
      const float f = data[(size_t)ex * g.sites + s] / t.nw[i].w;
      store_pop(pop, g, i, z, y, x, from_f<ST>(fmaf(f, ri, -1.f)));
    }
    return;
  }
  for (int i = 0; i < Ni; ++i) {
    const bool inert = __float_as_int(t.au[i].w) & 8;
    store_pop(pop, g, i, z, y, x, from_f<ST>(inert ? 0.f : fmaf(f_of(i), ri, -1.f)));
  }
}

template <class ST>
__device__ __forceinline__ float f_at(const ST* pop, const float* e, const Grid& g, int i, int z,
                                      int y, int x) {
  const float Eh = e[eidx(g, z, y, x)];
  return fmaf(Eh, to_f<ST>(pop[pidx(g, i, z, y, x)]), Eh);
}

template <class ST>
__global__ void k_moments16(Grid g, int N, const ST* __restrict__ pop, const float* __restrict__ e,
                            float* __restrict__ E, float* __restrict__ F, float* __restrict__ P,
                            DirTable t) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.sites) return;
  int x, y, z;
  site_xyz(g, s, x, y, z);
  const float Eh = e[eidx(g, z, y, x)];
  float es = 0, fx = 0, fy = 0, fz = 0, pxx = 0, pxy = 0, pxz = 0, pyy = 0, pyz = 0, pzz = 0;
  for (int i = 0; i < N; ++i) {
    const float4 nw = t.nw[i];
    const float v = nw.w * fmaf(Eh, to_f<ST>(pop[pidx(g, i, z, y, x)]), Eh);
    es += v;
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
  if (E) E[s] = es;
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

template <class ST>
__global__ void k_decode16(Grid g, int Next, const int* __restrict__ int_of_ext,
                           const ST* __restrict__ pop, const float* __restrict__ e,
                           float* __restrict__ out, DirTable t) {
  const long long total = g.sites * (long long)Next;
  for (long long k = blockIdx.x * (long long)blockDim.x + threadIdx.x; k < total;
       k += (long long)gridDim.x * blockDim.x) {
    const int ex = (int)(k / g.sites);
    int x, y, z;
    site_xyz(g, k % g.sites, x, y, z);
    const int i = int_of_ext[ex];
    out[k] = t.nw[i].w * f_at(pop, e, g, i, z, y, x);
  }
}

// Frozen cells in 16-bit storage: the site's E^ becomes the sum of the
// prescribed values and every direction is re-encoded against it.
template <class ST>
__global__ void k_frozen16(Grid g, int Ni, int Next, const int* __restrict__ int_of_ext, int ncells,
                           const int64_t* __restrict__ cells, const float* __restrict__ vals,
                           ST* __restrict__ pop, float* __restrict__ e, double* injection,
                           DirTable t) {
  const int c = blockIdx.x * blockDim.x + threadIdx.x;
  if (c >= ncells) return;
  int x, y, z;
  site_xyz(g, cells[c], x, y, z);
  double old = 0.0, neu = 0.0;
  for (int i = 0; i < Ni; ++i) old += (double)(t.nw[i].w * f_at(pop, e, g, i, z, y, x));
  float E = 0.f;
  for (int ex = 0; ex < Next; ++ex) {
    E += vals[(size_t)c * Next + ex];
    neu += (double)vals[(size_t)c * Next + ex];
  }
  const float Eh = fmaxf(E, EPS_E);
  const float ri = 1.f / Eh;
  for (int ex = 0; ex < Next; ++ex) {
    const int i = int_of_ext[ex];
    const float f = vals[(size_t)c * Next + ex] / t.nw[i].w;
    store_pop(pop, g, i, z, y, x, from_f<ST>(fmaf(f, ri, -1.f)));
  }
  store_e_site(e, g, z, y, x, Eh);
  if (injection) atomicAdd(injection, neu - old);
}

template <class ST>
__global__ void k_total_partials16(Grid g, int N, const ST* __restrict__ pop,
                                   const float* __restrict__ e, double* __restrict__ partials,
                                   DirTable t) {
  __shared__ double sh[BLK];
  double acc = 0.0;
  for (long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x; s < g.sites;
       s += (long long)gridDim.x * blockDim.x) {
    int x, y, z;
    site_xyz(g, s, x, y, z);
    float v = 0.f;
    for (int i = 0; i < N; ++i) v = fmaf(t.nw[i].w, f_at(pop, e, g, i, z, y, x), v);
    acc += (double)v;
  }
  sh[threadIdx.x] = acc;
  __syncthreads();
  for (int w = blockDim.x / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) sh[threadIdx.x] += sh[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partials[blockIdx.x] = sh[0];
}

// Coupling outputs (Sec. 5, coupling step 4): from the site's E, F, P and
// the fluid velocity v, the comoving J = W^2 (E - 2 F.v + P:vv) (Eq. J),
// H_j = W^3 (F.v - E) v_j + W h_ji F^i - W h_ji v_k P^ik with
// h_ij = W^2 v_i v_j + delta_ij, and S_0 = W (kt_a J - eta_t) + kt H^0,
// S_j = W (kt_a J - eta_t) v_j + kt H_j with kt = kt_a + kt_0 (kt_1 = 0):
// the lab components of the four-vector (kt_a J - eta_t) u^mu + kt H^mu, with
// H^0 = v.H the time component of the comoving flux (H^mu u_mu = 0,
// signature -+++).  ST = float: populations; 16-bit types: the deviation
// form against the E array `e`.
template <class ST>
__global__ void k_coupling(Grid g, int N, const ST* __restrict__ pop, const float* __restrict__ e,
                           DirTable t, MovingCoef c, float* __restrict__ Jo, float* __restrict__ Ho,
                           float* __restrict__ So) {
  const long long s = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (s >= g.sites) return;
  int x, y, z;
  site_xyz(g, s, x, y, z);
  float Eh = 0.f;
  if (!std::is_same<ST, float>::value) Eh = e[eidx(g, z, y, x)];
  float E = 0, Fx = 0, Fy = 0, Fz = 0, Pxx = 0, Pxy = 0, Pxz = 0, Pyy = 0, Pyz = 0, Pzz = 0;
  for (int i = 0; i < N; ++i) {
    const float4 nw = t.nw[i];
    float I;
    if constexpr (std::is_same<ST, float>::value) I = pop[pidx(g, i, z, y, x)];
    else I = nw.w * fmaf(Eh, to_f<ST>(pop[pidx(g, i, z, y, x)]), Eh);
    E += I;
    Fx = fmaf(nw.x, I, Fx);
    Fy = fmaf(nw.y, I, Fy);
    Fz = fmaf(nw.z, I, Fz);
    Pxx = fmaf(nw.x * nw.x, I, Pxx);
    Pxy = fmaf(nw.x * nw.y, I, Pxy);
    Pxz = fmaf(nw.x * nw.z, I, Pxz);
    Pyy = fmaf(nw.y * nw.y, I, Pyy);
    Pyz = fmaf(nw.y * nw.z, I, Pyz);
    Pzz = fmaf(nw.z * nw.z, I, Pzz);
  }
  const float vx = c.v ? c.v[s] : 0.f, vy = c.v ? c.v[g.sites + s] : 0.f,
              vz = c.v ? c.v[2 * g.sites + s] : 0.f;
  const float W2 = 1.f / (1.f - (vx * vx + vy * vy + vz * vz));
  const float W = sqrtf(W2);
  const float Fv = Fx * vx + Fy * vy + Fz * vz;
  // Pv_i = P^ik v_k
  const float Pvx = Pxx * vx + Pxy * vy + Pxz * vz;
  const float Pvy = Pxy * vx + Pyy * vy + Pyz * vz;
  const float Pvz = Pxz * vx + Pyz * vy + Pzz * vz;
  const float Pvv = Pvx * vx + Pvy * vy + Pvz * vz;
  const float J = W2 * (E - 2.f * Fv + Pvv);
  // h_ji a^i = a_j + W^2 v_j (v.a) for a = F - Pv
  const float ax = Fx - Pvx, ay = Fy - Pvy, az = Fz - Pvz;
  const float va = vx * ax + vy * ay + vz * az;
  const float c1 = W * W2 * (Fv - E), c2 = W * W2 * va;
  const float Hx = c1 * vx + W * ax + c2 * vx;
  const float Hy = c1 * vy + W * ay + c2 * vy;
  const float Hz = c1 * vz + W * az + c2 * vz;
  if (Jo) Jo[s] = J;
  if (Ho) {
    Ho[s] = Hx;
    Ho[g.sites + s] = Hy;
    Ho[2 * g.sites + s] = Hz;
  }
  if (So) {
    const float kta = c.kta ? c.kta[s] : c.kta_s, kt0 = c.kt0 ? c.kt0[s] : c.kt0_s;
    const float etat = c.etat ? c.etat[s] : c.etat_s;
    const float kt = kta + kt0;
    // time component of the comoving flux four-vector, H^mu u_mu = 0
    const float H0 = vx * Hx + vy * Hy + vz * Hz;
    const float emit = W * (kta * J - etat);
    So[s] = fmaf(kt, H0, emit);
    So[g.sites + s] = fmaf(kt, Hx, emit * vx);
    So[2 * g.sites + s] = fmaf(kt, Hy, emit * vy);
    So[3 * g.sites + s] = fmaf(kt, Hz, emit * vz);
  }
}

unsigned grid1d(long long n) { return (unsigned)((n + BLK - 1) / BLK); }

}  // namespace

cudaError_t launch_init_state(const Grid& g, int Ni, int Next, const int* int_of_ext,
                              const float* data, int kind, void* pop, float* e, int storage,
                              const DirTable& t, cudaStream_t s) {
  if (storage == ST_F32)
    k_init_state<<<grid1d(g.sites), BLK, 0, s>>>(g, Ni, Next, int_of_ext, data, kind,
                                                 static_cast<float*>(pop), t);
  else if (storage == ST_F16)
    k_init_state16<__half><<<grid1d(g.sites), BLK, 0, s>>>(g, Ni, Next, int_of_ext, data, kind,
                                                           static_cast<__half*>(pop), e, t);
  else
    k_init_state16<__nv_bfloat16><<<grid1d(g.sites), BLK, 0, s>>>(
        g, Ni, Next, int_of_ext, data, kind, static_cast<__nv_bfloat16*>(pop), e, t);
  return cudaGetLastError();
}

cudaError_t launch_moments(const Grid& g, int N, const void* pop, const float* e, int storage,
                           const DirTable& t, float* E, float* F, float* P, cudaStream_t s) {
  if (storage == ST_F32)
    k_moments<<<grid1d(g.sites), BLK, 0, s>>>(g, N, pop, E, F, P, t);
  else if (storage == ST_F16)
    k_moments16<__half><<<grid1d(g.sites), BLK, 0, s>>>(g, N, static_cast<const __half*>(pop), e,
                                                        E, F, P, t);
  else
    k_moments16<__nv_bfloat16><<<grid1d(g.sites), BLK, 0, s>>>(
        g, N, static_cast<const __nv_bfloat16*>(pop), e, E, F, P, t);
  return cudaGetLastError();
}

cudaError_t launch_decode(const Grid& g, int Next, const int* int_of_ext, const void* pop,
                          const float* e, int storage, const DirTable& t, float* out,
                          cudaStream_t s) {
  if (storage == ST_F32)
    k_decode<<<1024, BLK, 0, s>>>(g, Next, int_of_ext, pop, out);
  else if (storage == ST_F16)
    k_decode16<__half><<<1024, BLK, 0, s>>>(g, Next, int_of_ext, static_cast<const __half*>(pop),
                                            e, out, t);
  else
    k_decode16<__nv_bfloat16><<<1024, BLK, 0, s>>>(
        g, Next, int_of_ext, static_cast<const __nv_bfloat16*>(pop), e, out, t);
  return cudaGetLastError();
}

cudaError_t launch_frozen(const Grid& g, int Ni, int Next, const int* int_of_ext, int ncells,
                          const int64_t* cells, const float* vals, void* pop, float* e,
                          int storage, const DirTable& t, double* injection_acc, cudaStream_t s) {
  if (ncells <= 0) return cudaSuccess;
  const int nb = (ncells + BLK - 1) / BLK;
  if (storage == ST_F32)
    k_frozen<<<nb, BLK, 0, s>>>(g, Next, int_of_ext, ncells, cells, vals,
                                static_cast<float*>(pop), injection_acc);
  else if (storage == ST_F16)
    k_frozen16<__half><<<nb, BLK, 0, s>>>(g, Ni, Next, int_of_ext, ncells, cells, vals,
                                          static_cast<__half*>(pop), e, injection_acc, t);
  else
    k_frozen16<__nv_bfloat16><<<nb, BLK, 0, s>>>(g, Ni, Next, int_of_ext, ncells, cells, vals,
                                                 static_cast<__nv_bfloat16*>(pop), e,
                                                 injection_acc, t);
  return cudaGetLastError();
}

cudaError_t launch_coupling(const Grid& g, int N, const void* pop, const float* e, int storage,
                            const DirTable& t, const MovingCoef& c, float* J, float* H, float* S,
                            cudaStream_t s) {
  if (storage == ST_F32)
    k_coupling<float><<<grid1d(g.sites), BLK, 0, s>>>(g, N, static_cast<const float*>(pop), e, t,
                                                      c, J, H, S);
  else if (storage == ST_F16)
    k_coupling<__half><<<grid1d(g.sites), BLK, 0, s>>>(g, N, static_cast<const __half*>(pop), e,
                                                       t, c, J, H, S);
  else
    k_coupling<__nv_bfloat16><<<grid1d(g.sites), BLK, 0, s>>>(
        g, N, static_cast<const __nv_bfloat16*>(pop), e, t, c, J, H, S);
  return cudaGetLastError();
}

cudaError_t launch_budget_finalize(const double* partials, int nblocks, double* acc,
                                   cudaStream_t s) {
  k_budget_finalize<<<1, BLK, 0, s>>>(partials, nblocks, acc);
  return cudaGetLastError();
}

cudaError_t launch_total_energy(const Grid& g, int N, const void* pop, const float* e, int storage,
                                const DirTable& t, double* partials, int max_blocks, double* out,
                                cudaStream_t s) {
  int nb = (int)std::min<long long>((long long)max_blocks, (long long)grid1d(g.sites));
  if (nb < 1) nb = 1;
  if (storage == ST_F32)
    k_total_partials<<<nb, BLK, 0, s>>>(g, N, pop, partials);
  else if (storage == ST_F16)
    k_total_partials16<__half><<<nb, BLK, 0, s>>>(g, N, static_cast<const __half*>(pop), e,
                                                  partials, t);
  else
    k_total_partials16<__nv_bfloat16><<<nb, BLK, 0, s>>>(
        g, N, static_cast<const __nv_bfloat16*>(pop), e, partials, t);
  k_sum_partials<<<1, BLK, 0, s>>>(partials, nb, out);
  return cudaGetLastError();
}

}  // namespace lbrt
