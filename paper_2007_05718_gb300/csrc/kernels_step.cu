// Fused stream + collide kernels for the grey radiative LB step
// (Weih et al. 2020, Sec. 3.3; moving fluid: App. B).
//
// One thread owns one lattice site and a group of DPT directions; the
// blockDim.z = G groups of a CTA together cover all N directions of the
// CTA's 32 x TY sites.  Per direction the thread pulls the streamed value
// I*_i(r) from the 2^d upwind corners of Eq. (interp) and keeps it in a
// register; the per-site partial sums of the G groups meet in shared
// memory; the site-local implicit collision is then closed-form and every
// output population is written once.
#include "lb_rt_internal.h"

namespace lbrt {

namespace {

constexpr int TY = 4;  // sites per CTA along y (32 along x)

// Upwind neighbours of one site: linear offsets of the -1 / +1 neighbour
// along x, y, z and whether it exists (a vacuum face reads zero).
struct Site {
  int site;
  int om[3], op[3];
  bool km[3], kp[3];
};

__device__ __forceinline__ void neighbour(int c, int n, int stride, int periodic, int& off_m,
                                          int& off_p, bool& ok_m, bool& ok_p) {
  ok_m = (c > 0) || periodic;
  ok_p = (c < n - 1) || periodic;
  off_m = (c > 0) ? -stride : (periodic ? (n - 1) * stride : 0);
  off_p = (c < n - 1) ? stride : (periodic ? -(n - 1) * stride : 0);
}

__device__ __forceinline__ Site make_site(const Grid& g, int x, int y, int z) {
  Site s;
  s.site = (z * g.ny + y) * g.nx + x;
  neighbour(x, g.nx, 1, g.periodic[0], s.om[0], s.op[0], s.km[0], s.kp[0]);
  neighbour(y, g.ny, g.nx, g.periodic[1], s.om[1], s.op[1], s.km[1], s.kp[1]);
  neighbour(z, g.nz, g.nx * g.ny, g.periodic[2], s.om[2], s.op[2], s.km[2], s.kp[2]);
  return s;
}

// I*_i(r) of Eq. (interp): corners r - b o sgn(n_i), weights prod_a
// (b_a a_a + (1 - b_a)(1 - a_a)), evaluated as nested linear interpolations
// (x, then y, then z).  `p` points at I_i(r).
__device__ __forceinline__ float pull(const float* __restrict__ p, const Site& s, float4 au) {
  const int oct = __float_as_int(au.w);
  const int dxo = (oct & 1) ? s.op[0] : s.om[0];
  const int dyo = (oct & 2) ? s.op[1] : s.om[1];
  const int dzo = (oct & 4) ? s.op[2] : s.om[2];
  const float vx = ((oct & 1) ? s.kp[0] : s.km[0]) ? 1.f : 0.f;
  const float vy = ((oct & 2) ? s.kp[1] : s.km[1]) ? 1.f : 0.f;
  const float vz = ((oct & 4) ? s.kp[2] : s.km[2]) ? 1.f : 0.f;
  const float ax = au.x, ay = au.y, az = au.z;
  const float v000 = __ldg(p);
  const float v100 = vx * __ldg(p + dxo);
  const float v010 = vy * __ldg(p + dyo);
  const float v110 = vx * vy * __ldg(p + dxo + dyo);
  const float b0 = fmaf(ax, v100 - v000, v000);
  const float b1 = fmaf(ax, v110 - v010, v010);
  const float r0 = fmaf(ay, b1 - b0, b0);
  if (az == 0.f) return r0;
  const float v001 = vz * __ldg(p + dzo);
  const float v101 = vz * vx * __ldg(p + dzo + dxo);
  const float v011 = vz * vy * __ldg(p + dzo + dyo);
  const float v111 = vz * vx * vy * __ldg(p + dzo + dxo + dyo);
  const float c0 = fmaf(ax, v101 - v001, v001);
  const float c1 = fmaf(ax, v111 - v011, v011);
  const float r1 = fmaf(ay, c1 - c0, c0);
  return fmaf(az, r1 - r0, r0);
}

// Site scalars of the static collision such that
//   I_i^{n+1} = alpha I*_i + w_i (c0 + n_i . c1).
//   implicit exact (Eq. rte_implicit, isotropic table), A = 1/(1 + dt (k0 + ka)):
//     E = (E* + dt eta) / (1 + dt ka),  F = F* / (1 + dt (ka + k0) - dt k0 lam / d),
//     alpha = A, c0 = A dt (eta + k0 E), c1 = A dt k0 lam F;
//   explicit (Eq. collision-step): alpha = 1 - dt (k0 + ka),
//     c0 = dt (k0 E* + eta), c1 = dt k0 lam F*;
//   Lambda-K (Sec. 3.3): K passes started from (E*, F*); for an isotropic
//     table a pass maps (E, F) -> (A (E* + dt eta + dt k0 E), A (F* + dt k0 lam F / d)),
//     and the output populations are those of pass K, built from the
//     moments of pass K - 1.
struct Coll {
  float alpha, c0, c1x, c1y, c1z;
  float Enew;  // energy of the output populations (up to rounding)
};

__device__ __forceinline__ Coll collision_coefficients(int mode, int iters, float dt, float inv_d,
                                                       float ka, float k0, float lam, float eta,
                                                       float Es, float Fx, float Fy, float Fz) {
  Coll c;
  if (mode == LB_RT_EXPLICIT) {
    // c0 = dt (k0 E* + eta) is taken as E_new - alpha E* with
    // E_new = E* + dt (eta - ka E*), so that the site energy the outputs sum to
    // carries no systematic rounding bias of alpha (pure scattering: E_new = E*).
    c.alpha = 1.f - dt * (k0 + ka);
    c.Enew = fmaf(dt, eta - ka * Es, Es);
    c.c0 = fmaf(-c.alpha, Es, c.Enew);
    const float g = dt * k0 * lam;
    c.c1x = g * Fx; c.c1y = g * Fy; c.c1z = g * Fz;
    return c;
  }
  const float A = 1.f / (1.f + dt * (k0 + ka));
  float E, gx, gy, gz;
  if (mode == LB_RT_LAMBDA_K) {
    E = Es; gx = Fx; gy = Fy; gz = Fz;
    const float q = dt * k0 * lam * inv_d;
    for (int m = 1; m < iters; ++m) {
      E = A * (Es + dt * eta + dt * k0 * E);
      gx = A * (Fx + q * gx); gy = A * (Fy + q * gy); gz = A * (Fz + q * gz);
    }
    c.alpha = A;
    c.c0 = A * dt * (eta + k0 * E);
    c.Enew = fmaf(A, Es, c.c0);
  } else {
    // exact step: c0 = A dt (eta + k0 E) equals E - A E*, and that residual
    // form keeps sum_i I_i^{n+1} = E free of a systematic float32 bias in A
    // (pure scattering: E = E* exactly, so energy is conserved to rounding).
    E = (Es + dt * eta) / (1.f + dt * ka);
    const float r = 1.f / (1.f + dt * (ka + k0) - dt * k0 * lam * inv_d);
    gx = Fx * r; gy = Fy * r; gz = Fz * r;
    c.alpha = A;
    c.c0 = fmaf(-A, Es, E);
    c.Enew = E;
  }
  const float g = A * dt * k0 * lam;
  c.c1x = g * gx; c.c1y = g * gy; c.c1z = g * gz;
  return c;
}

__device__ __forceinline__ float field(const float* __restrict__ p, float s, long long i) {
  return p ? __ldg(p + i) : s;
}

// FP64 per-CTA sums (sum E*, sum E_collided) for the energy budget.
__device__ __forceinline__ void budget_add(double* partials, double a, double b) {
  for (int s = 16; s > 0; s >>= 1) {
    a += __shfl_xor_sync(0xffffffffu, a, s);
    b += __shfl_xor_sync(0xffffffffu, b, s);
  }
  if (threadIdx.x == 0) {
    const long long blk =
        ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
    atomicAdd(partials + 2 * blk, a);
    atomicAdd(partials + 2 * blk + 1, b);
  }
}

template <int DPT>
__global__ void __launch_bounds__(32 * TY * 4)
k_step_static_f32(const StepLaunch L, const StaticCoef cf, const DirTable t) {
  extern __shared__ float4 red[];  // [G][TY*32]
  const int G = blockDim.z;
  const int tx = threadIdx.x, ty = threadIdx.y, g = threadIdx.z;
  const int x = blockIdx.x * 32 + tx, y = blockIdx.y * TY + ty, z = blockIdx.z;
  const bool valid = (x < L.g.nx) && (y < L.g.ny);
  const Site S = make_site(L.g, valid ? x : 0, valid ? y : 0, z);
  const long long sites = L.g.sites;
  const float* __restrict__ in = static_cast<const float*>(L.in);
  float* __restrict__ out = static_cast<float*>(L.out);

  const int i0 = g * DPT;
  const int nd = min(DPT, L.N - i0);
  float Is[DPT];
  float e = 0.f, fx = 0.f, fy = 0.f, fz = 0.f;
#pragma unroll
  for (int k = 0; k < DPT; ++k) {
    Is[k] = 0.f;
    if (k < nd) {
      const float4 nw = t.nw[i0 + k];
      const float r = pull(in + (size_t)(i0 + k) * sites + S.site, S, t.au[i0 + k]);
      Is[k] = r;
      e += r;
      fx = fmaf(nw.x, r, fx);
      fy = fmaf(nw.y, r, fy);
      fz = fmaf(nw.z, r, fz);
    }
  }
  const int sid = ty * 32 + tx;
  red[g * (TY * 32) + sid] = make_float4(e, fx, fy, fz);
  __syncthreads();
  float4 m = red[sid];
  for (int gg = 1; gg < G; ++gg) {
    const float4 q = red[gg * (TY * 32) + sid];
    m.x += q.x; m.y += q.y; m.z += q.z; m.w += q.w;
  }
  const float ka = field(cf.ka, cf.ka_s, S.site), k0 = field(cf.k0, cf.k0_s, S.site);
  const float lam = field(cf.lam, cf.lam_s, S.site), eta = field(cf.eta, cf.eta_s, S.site);
  const float inv_d = 1.f / (float)L.g.dims;
  const Coll c = collision_coefficients(L.collision, L.lambda_iters, L.dt, inv_d, ka, k0, lam,
                                        eta, m.x, m.y, m.z, m.w);
  if (valid) {
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      if (k < nd) {
        const float4 nw = t.nw[i0 + k];
        out[(size_t)(i0 + k) * sites + S.site] =
            fmaf(c.alpha, Is[k], nw.w * (c.c0 + fmaf(nw.x, c.c1x, fmaf(nw.y, c.c1y, nw.z * c.c1z))));
      }
    }
  }
  if (L.budget_partials && g == 0)
    budget_add(L.budget_partials, valid ? (double)m.x : 0.0, valid ? (double)c.Enew : 0.0);
}

// Mixed-frame moving fluid (App. B), exact implicit step.  Per site
// W = 1/sqrt(1 - v^2); per direction beta_i = 1 - v.n_i,
// A_i = 1/(1 + dt W beta_i (kt_a + kt_0)), D_i = (W beta_i)^-3, and with
// g_i = A_i dt w_i D_i:
//   I_i^{n+1} = A_i I*_i + g_i (eta_t + kt_0 J),
//   J = W^2 sum beta_i^2 I_i^{n+1} = X / (1 - Y),
//   X = W^2 sum beta_i^2 (A_i I*_i + g_i eta_t),  Y = kt_0 W^2 sum beta_i^2 g_i.
template <int DPT>
__global__ void __launch_bounds__(32 * TY * 4)
k_step_moving_f32(const StepLaunch L, const MovingCoef cf, const DirTable t) {
  extern __shared__ float4 red[];  // [2][G][TY*32]
  const int G = blockDim.z;
  const int tx = threadIdx.x, ty = threadIdx.y, g = threadIdx.z;
  const int x = blockIdx.x * 32 + tx, y = blockIdx.y * TY + ty, z = blockIdx.z;
  const bool valid = (x < L.g.nx) && (y < L.g.ny);
  const Site S = make_site(L.g, valid ? x : 0, valid ? y : 0, z);
  const long long sites = L.g.sites;
  const float* __restrict__ in = static_cast<const float*>(L.in);
  float* __restrict__ out = static_cast<float*>(L.out);

  float vx = 0.f, vy = 0.f, vz = 0.f;
  if (cf.v) {
    vx = __ldg(cf.v + S.site);
    vy = __ldg(cf.v + sites + S.site);
    vz = __ldg(cf.v + 2 * sites + S.site);
  }
  const float kta = field(cf.kta, cf.kta_s, S.site), kt0 = field(cf.kt0, cf.kt0_s, S.site);
  const float etat = field(cf.etat, cf.etat_s, S.site);
  const float W = rsqrtf(1.f - (vx * vx + vy * vy + vz * vz));
  const float W2 = W * W;
  const float dt = L.dt;
  const float ksum = kta + kt0;

  const int i0 = g * DPT;
  const int nd = min(DPT, L.N - i0);
  float AI[DPT], gi[DPT];
  float es = 0.f, X = 0.f, Y = 0.f, S1 = 0.f, S2 = 0.f;
#pragma unroll
  for (int k = 0; k < DPT; ++k) {
    AI[k] = 0.f;
    gi[k] = 0.f;
    if (k < nd) {
      const float4 nw = t.nw[i0 + k];
      const float r = pull(in + (size_t)(i0 + k) * sites + S.site, S, t.au[i0 + k]);
      const float beta = 1.f - fmaf(vx, nw.x, fmaf(vy, nw.y, vz * nw.z));
      const float Wb = W * beta;
      const float A = 1.f / fmaf(dt * Wb, ksum, 1.f);
      const float iWb = 1.f / Wb;
      const float gg = A * dt * nw.w * (iWb * iWb * iWb);
      const float ai = A * r;
      const float b2 = beta * beta;
      AI[k] = ai;
      gi[k] = gg;
      es += r;
      X = fmaf(b2, fmaf(gg, etat, ai), X);
      Y = fmaf(b2, gg, Y);
      S1 += ai;
      S2 += gg;
    }
  }
  const int sid = ty * 32 + tx;
  red[g * (TY * 32) + sid] = make_float4(es, X, Y, S1);
  red[(G + g) * (TY * 32) + sid] = make_float4(S2, 0.f, 0.f, 0.f);
  __syncthreads();
  float4 m = red[sid];
  float s2 = red[G * (TY * 32) + sid].x;
  for (int q = 1; q < G; ++q) {
    const float4 a = red[q * (TY * 32) + sid];
    m.x += a.x; m.y += a.y; m.z += a.z; m.w += a.w;
    s2 += red[(G + q) * (TY * 32) + sid].x;
  }
  const float J = (W2 * m.y) / (1.f - kt0 * W2 * m.z);
  const float src = fmaf(kt0, J, etat);
  if (valid) {
#pragma unroll
    for (int k = 0; k < DPT; ++k)
      if (k < nd) out[(size_t)(i0 + k) * sites + S.site] = fmaf(gi[k], src, AI[k]);
  }
  if (L.budget_partials && g == 0)
    budget_add(L.budget_partials, valid ? (double)m.x : 0.0,
               valid ? (double)fmaf(s2, src, m.w) : 0.0);
}

int groups_for(int N, int* per) {
  const int G = (N + 47) / 48;
  *per = (N + G - 1) / G;
  return G;
}

template <int DPT, bool MOVING, class Coef>
cudaError_t launch_f32(const StepLaunch& L, const Coef& c, const DirTable& t, int G,
                       cudaStream_t s, int* nblocks) {
  dim3 block(32, TY, G);
  dim3 grid((L.g.nx + 31) / 32, (L.g.ny + TY - 1) / TY, L.g.nz);
  if (nblocks) *nblocks = grid.x * grid.y * grid.z;
  if constexpr (MOVING) {
    k_step_moving_f32<DPT><<<grid, block, sizeof(float4) * 2 * G * TY * 32, s>>>(L, c, t);
  } else {
    k_step_static_f32<DPT><<<grid, block, sizeof(float4) * G * TY * 32, s>>>(L, c, t);
  }
  return cudaGetLastError();
}

template <bool MOVING, class Coef>
cudaError_t dispatch(const StepLaunch& L, const Coef& c, const DirTable& t, int storage,
                     cudaStream_t s, int* nblocks) {
  if (storage != ST_F32) return cudaErrorNotSupported;
  int per = 0;
  const int G = groups_for(L.N, &per);
  if (G > 4 || L.N < 1) return cudaErrorInvalidValue;
  if (per <= 16) return launch_f32<16, MOVING>(L, c, t, G, s, nblocks);
  if (per <= 32) return launch_f32<32, MOVING>(L, c, t, G, s, nblocks);
  return launch_f32<48, MOVING>(L, c, t, G, s, nblocks);
}

}  // namespace

cudaError_t launch_step_static(const StepLaunch& L, const StaticCoef& c, const DirTable& t,
                               int storage, cudaStream_t s, int* nblocks) {
  return dispatch<false>(L, c, t, storage, s, nblocks);
}

cudaError_t launch_step_moving(const StepLaunch& L, const MovingCoef& c, const DirTable& t,
                               int storage, cudaStream_t s, int* nblocks) {
  return dispatch<true>(L, c, t, storage, s, nblocks);
}

}  // namespace lbrt
