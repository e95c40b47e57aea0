// Fused stream + collide kernel for a moving background fluid (mixed-frame
// equation of Weih et al. 2020, App. B; streaming of Sec. 3.3), and the
// step-kernel dispatch.
//
// One thread owns one lattice site and a group of DPT directions; the
// blockDim.z = G groups of a CTA together cover all N directions of the
// CTA's 32 x TY sites.  Per direction the thread pulls the streamed value
// I*_i(r) from the 2^d upwind corners of Eq. (interp) (the padded layout's
// ghost layer supplies periodic images and vacuum zeros) and keeps the
// per-direction collision terms in registers; the per-site sums of the G
// groups meet in shared memory and the site-local implicit collision is
// closed-form.
#include <type_traits>

#include "lb_rt_internal.h"

namespace lbrt {

cudaError_t launch_tma_static(const StepLaunch& L, const StaticCoef& c, const DirTable& t,
                              int dpt, int zc, cudaStream_t s, int* nblocks);

namespace {

constexpr int TY = 4;  // sites per CTA along y (32 along x)

// I*_i(r) of Eq. (interp): corners r - b o sgn(n_i), weights prod_a
// (b_a a_a + (1 - b_a)(1 - a_a)), evaluated as nested linear interpolations
// (x, then y, then z).  `p` points at I_i(r) in the padded layout.
__device__ __forceinline__ float pull(const float* __restrict__ p, const Grid& g, float4 au) {
  const int oct = __float_as_int(au.w);
  const long long dxo = (oct & 1) ? 1 : -1;
  const long long dyo = (oct & 2) ? g.sy : -g.sy;
  const long long dzo = (oct & 4) ? g.sz : -g.sz;
  const float ax = au.x, ay = au.y, az = au.z;
  const float v000 = __ldg(p);
  const float v100 = __ldg(p + dxo);
  const float v010 = __ldg(p + dyo);
  const float v110 = __ldg(p + dxo + dyo);
  const float b0 = fmaf(ax, v100 - v000, v000);
  const float b1 = fmaf(ax, v110 - v010, v010);
  const float r0 = fmaf(ay, b1 - b0, b0);
  if (az == 0.f) return r0;
  const float v001 = __ldg(p + dzo);
  const float v101 = __ldg(p + dzo + dxo);
  const float v011 = __ldg(p + dzo + dyo);
  const float v111 = __ldg(p + dzo + dxo + dyo);
  const float c0 = fmaf(ax, v101 - v001, v001);
  const float c1 = fmaf(ax, v111 - v011, v011);
  const float r1 = fmaf(ay, c1 - c0, c0);
  return fmaf(az, r1 - r0, r0);
}

// 16-bit storage (f_i = I_i / w_i = E^ (1 + q_i), E^ in a padded float32
// array): the streamed f*_i of Eq. (interp) from the decoded corners.  `q`
// points at q_i(r), `e` at E^(r).
__device__ __forceinline__ float to_f32(float v) { return v; }
__device__ __forceinline__ float to_f32(__half v) { return __half2float(v); }
__device__ __forceinline__ float to_f32(__nv_bfloat16 v) { return __bfloat162float(v); }

template <class ST>
__device__ __forceinline__ float pull16(const ST* __restrict__ q, const float* __restrict__ e,
                                        const Grid& g, float4 au) {
  const int oct = __float_as_int(au.w);
  const long long dxo = (oct & 1) ? 1 : -1;
  const long long dyo = (oct & 2) ? g.sy : -g.sy;
  const long long dzo = (oct & 4) ? g.sz : -g.sz;
  const long long eyo = (oct & 2) ? g.PX : -(long long)g.PX;
  const long long ezo = (oct & 4) ? (long long)g.PX * g.PY : -(long long)g.PX * g.PY;
  auto f = [&](long long dq, long long de) {
    const float E = __ldg(e + de);
    return fmaf(E, to_f32(q[dq]), E);
  };
  const float ax = au.x, ay = au.y, az = au.z;
  const float v000 = f(0, 0), v100 = f(dxo, dxo), v010 = f(dyo, eyo), v110 = f(dxo + dyo, dxo + eyo);
  const float b0 = fmaf(ax, v100 - v000, v000);
  const float b1 = fmaf(ax, v110 - v010, v010);
  const float r0 = fmaf(ay, b1 - b0, b0);
  if (az == 0.f) return r0;
  const float v001 = f(dzo, ezo), v101 = f(dzo + dxo, ezo + dxo), v011 = f(dzo + dyo, ezo + eyo),
              v111 = f(dzo + dxo + dyo, ezo + dxo + eyo);
  const float c0 = fmaf(ax, v101 - v001, v001);
  const float c1 = fmaf(ax, v111 - v011, v011);
  const float r1 = fmaf(ay, c1 - c0, c0);
  return fmaf(az, r1 - r0, r0);
}

template <class ST> __device__ __forceinline__ ST from_f32(float v);
template <> __device__ __forceinline__ __half from_f32<__half>(float v) { return __float2half_rn(v); }
template <> __device__ __forceinline__ __nv_bfloat16 from_f32<__nv_bfloat16>(float v) {
  return __float2bfloat16_rn(v);
}

// E^ of a site into the padded E array and its periodic mirrors.
__device__ __forceinline__ void store_e_mirrored(float* e, const Grid& g, int z, int y, int x,
                                                 float v) {
  int xs[3], ys[3], zs[3];
  const int nxs = mirrors(x, g.nx, g.periodic[0], GL, xs);
  const int nys = mirrors(y, g.ny, g.periodic[1], 1, ys);
  const int nzs = mirrors(z, g.nz, g.periodic[2], 1, zs);
  for (int a = 0; a < nzs; ++a)
    for (int b = 0; b < nys; ++b)
      for (int c = 0; c < nxs; ++c)
        e[(long long)zs[a] * g.PX * g.PY + (long long)ys[b] * g.PX + xs[c]] = v;
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

// Mixed-frame moving fluid (App. B), exact implicit step.  Per site
// W = 1/sqrt(1 - v^2); per direction beta_i = 1 - v.n_i,
// A_i = 1/(1 + dt W beta_i (kt_a + kt_0)), D_i = (W beta_i)^-3, and with
// g_i = A_i dt w_i D_i:
//   I_i^{n+1} = A_i I*_i + g_i (eta_t + kt_0 J),
//   J = W^2 sum beta_i^2 I_i^{n+1} = X / (1 - Y),
//   X = W^2 sum beta_i^2 (A_i I*_i + g_i eta_t),  Y = kt_0 W^2 sum beta_i^2 g_i.
// ST = float: populations I_i; ST = __half / __nv_bfloat16: the 16-bit
// deviation form, decoded at the corners and encoded against the site's new
// energy density E' = sum_i I_i^{n+1} = sum_i A_i I*_i + (eta_t + kt_0 J) sum_i g_i.
template <class ST, int DPT>
__global__ void __launch_bounds__(32 * TY * 4)
k_step_moving(const StepLaunch L, const MovingCoef cf, const DirTable t) {
  extern __shared__ float4 red[];  // [2][G][TY*32]
  const int G = blockDim.z;
  const int tx = threadIdx.x, ty = threadIdx.y, g = threadIdx.z;
  const Grid& gr = L.g;
  const int x = blockIdx.x * 32 + tx, y = blockIdx.y * TY + ty, z = blockIdx.z;
  const bool valid = (x < gr.nx) && (y < gr.ny);
  const int xs = valid ? x : 0, ys = valid ? y : 0;
  const long long site = ((long long)z * gr.ny + ys) * gr.nx + xs;
  const long long sites = gr.sites;
  const ST* __restrict__ in = static_cast<const ST*>(L.in);
  ST* __restrict__ out = static_cast<ST*>(L.out);
  constexpr bool F32 = std::is_same<ST, float>::value;

  float vx = 0.f, vy = 0.f, vz = 0.f;
  if (cf.v) {
    vx = __ldg(cf.v + site);
    vy = __ldg(cf.v + sites + site);
    vz = __ldg(cf.v + 2 * sites + site);
  }
  const float kta = field(cf.kta, cf.kta_s, site), kt0 = field(cf.kt0, cf.kt0_s, site);
  const float etat = field(cf.etat, cf.etat_s, site);
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
      float r;
      if constexpr (F32) {
        r = pull(in + pidx(gr, i0 + k, z, ys, xs), gr, t.au[i0 + k]);
      } else {
        const long long ei = (long long)(z + 1) * gr.PX * gr.PY + (long long)(ys + 1) * gr.PX + xs + GL;
        r = nw.w * pull16(in + pidx(gr, i0 + k, z, ys, xs), L.e_in + ei, gr, t.au[i0 + k]);
      }
      const float beta = 1.f - fmaf(vx, nw.x, fmaf(vy, nw.y, vz * nw.z));
      const float Wb = W * beta;
      // fast reciprocals (a few ulp): the denominators are >= 1 and
      // W beta >= W (1 - |v|) > 0
      const float A = __fdividef(1.f, fmaf(dt * Wb, ksum, 1.f));
      const float iWb = __fdividef(1.f, Wb);
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
    const bool mirror = has_mirror(gr, z, y, x);
    float rinv = 0.f;
    if constexpr (!F32) {
      const float Eh = fmaxf(fmaf(s2, src, m.w), 1e-30f);
      rinv = __fdividef(1.f, Eh);
      if (g == 0) store_e_mirrored(L.e_out, gr, z, y, x, Eh);
    }
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      if (k < nd) {
        const float o = fmaf(gi[k], src, AI[k]);
        ST v;
        if constexpr (F32) v = o;
        else v = from_f32<ST>(fmaf(__fdividef(o, t.nw[i0 + k].w), rinv, -1.f));
        if (mirror) store_pop(out, gr, i0 + k, z, y, x, v);
        else out[pidx(gr, i0 + k, z, y, x)] = v;
      }
    }
  }
  if (L.budget_partials && g == 0)
    budget_add(L.budget_partials, valid ? (double)m.x : 0.0,
               valid ? (double)fmaf(s2, src, m.w) : 0.0);
}

template <class ST, int DPT>
cudaError_t launch_moving(const StepLaunch& L, const MovingCoef& c, const DirTable& t, int G,
                          cudaStream_t s, int* nblocks) {
  dim3 block(32, TY, G);
  dim3 grid((L.g.nx + 31) / 32, (L.g.ny + TY - 1) / TY, L.g.nz);
  const long long nb_ = (long long)grid.x * grid.y * grid.z;
  if (L.budget_partials && nb_ > L.partials_cap) return cudaErrorInvalidValue;
  if (nblocks) *nblocks = (int)nb_;
  if (!std::is_same<ST, float>::value && (!L.e_in || !L.e_out)) return cudaErrorInvalidValue;
  k_step_moving<ST, DPT><<<grid, block, sizeof(float4) * 2 * G * TY * 32, s>>>(L, c, t);
  return cudaGetLastError();
}

}  // namespace

cudaError_t launch_step_static(const StepLaunch& L, const StaticCoef& c, const DirTable& t,
                               int storage, cudaStream_t s, int* nblocks) {
  if (L.sc) return launch_sc_static(L, c, t, storage, s, nblocks);
  if (storage != ST_F32) return launch_tma16_static(L, c, t, storage, s, nblocks);
  return launch_tma_static(L, c, t, L.dpt, L.zc, s, nblocks);
}

cudaError_t launch_step_moving(const StepLaunch& L, const MovingCoef& c, const DirTable& t,
                               int storage, cudaStream_t s, int* nblocks) {
  // FP32 with a tile plan: the TMA-fed kernel; otherwise one thread per site
  if (L.dpt > 0)
    return storage == ST_F32 ? launch_tma_moving(L, c, t, s, nblocks)
                             : launch_tma16_moving(L, c, t, storage, s, nblocks);
  const int N = L.N;
  const int G = (N + 47) / 48;
  if (G > 4 || N < 1) return cudaErrorInvalidValue;
  const int per = (N + G - 1) / G;
  auto go = [&](auto tag) {
    using ST = decltype(tag);
    if (per <= 16) return launch_moving<ST, 16>(L, c, t, G, s, nblocks);
    if (per <= 32) return launch_moving<ST, 32>(L, c, t, G, s, nblocks);
    return launch_moving<ST, 48>(L, c, t, G, s, nblocks);
  };
  if (storage == ST_F32) return go(float());
  if (storage == ST_F16) return go(__half());
  if (storage == ST_BF16) return go(__nv_bfloat16());
  return cudaErrorInvalidValue;
}

}  // namespace lbrt
