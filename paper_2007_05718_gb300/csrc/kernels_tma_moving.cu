// Fused stream + collide step for a moving background fluid, FP32
// populations, fed by TMA tensor tiles: the mixed-frame equation of Weih et
// al. 2020, App. B, with the streaming of Sec. 3.3 (Eq. interp).
//
// Tiles, boxes, the TMA ring and the z-sweep with the carried plane are those
// of the static kernel (kernels_tma.cu), one plane per batch.  The collision
// is per site and direction: with W = (1 - v^2)^(-1/2), beta_i = 1 - v.n_i,
//   A_i = 1 / (1 + dt W beta_i (kt_a + kt_0)),  g_i = A_i dt w_i (W beta_i)^-3,
//   I_i^{n+1} = A_i I*_i + g_i (eta_t + kt_0 J),
//   J = W^2 X / (1 - kt_0 W^2 Y),  X = sum beta_i^2 (A_i I*_i + g_i eta_t),
//   Y = sum beta_i^2 g_i.
// Each warp forms beta_i, A_i, g_i for its directions from the per-site
// fields held in registers and accumulates partial (sum I*, X, Y,
// sum A I*, sum g); coefficient units turn the CTA's sums into one scalar
// src = eta_t + kt_0 J per site; the output pass forms A_i and g_i again and
// stores A_i I*_i + g_i src.
#include <algorithm>

#include "lb_rt_internal.h"
#include "tma_common.cuh"

namespace lbrt {

namespace {

using namespace tma;

// Per-direction constants as pre-broadcast pairs: s0 = (a_x, a_x, a_y, a_y),
// s1 = (a_z', a_z', n_x, n_x), s2 = (n_y, n_y, n_z, n_z), s3 = (dt w, dt w,
// -, -); sh = offset of the x-upwind pair; inert = padding entry.
struct DirConstM {
  float4 s0, s1, s2, s3;
  int sh, inert, pad0, pad1;
};

constexpr int kQ = 5;  // partial quantities: sum I*, X, Y, sum A I*, sum g

__device__ __forceinline__ float2 f2rcp(float2 a) {
  return make_float2(__fdividef(1.f, a.x), __fdividef(1.f, a.y));
}

template <bool PER, int DPT, int R, int MAXT, int REGS>
__global__ void __launch_bounds__(MAXT) __maxnreg__(REGS)
k_step_moving_tma(const __grid_constant__ CUtensorMap tmap, const StepLaunch L,
                  const MovingCoef mc, const DirTable t) {
  constexpr int ZC = 1;
  constexpr int SLOT = slot_floats<DPT, ZC>();
  static_assert(SLOT >= kQ * 64, "the partial sums must fit in a consumed slot");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int G = blockDim.y;
  const int lane = threadIdx.x, g = threadIdx.y;
  const Grid& gr = L.g;
  const int nx = gr.nx, ny = gr.ny, nz = gr.nz;
  // shared layout: ring [G][R][SLOT] | src [64] | fields [2][6][64] |
  // dirs [N] | mbar [G][R] | budget [2][2] double | abort flag
  float* ring = reinterpret_cast<float*>(smem_raw);
  float* srcs = ring + (size_t)G * R * SLOT;
  // per-site fields (vx, vy, vz, kt_a, kt_0, eta_t) of the 64 sites of the
  // current item and of the next one, copied in by the last warp one item
  // ahead so that no warp waits on their global loads
  float* fbuf = srcs + 64;
  DirConstM* dirs = reinterpret_cast<DirConstM*>(fbuf + 2 * 6 * 64);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(dirs + G * DPT);
  double* bsum = reinterpret_cast<double*>(mbar + G * R);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bsum + 4);

  const int nxb = (nx + 63) / 64;
  const int ntiles = nxb * ny * L.nzc;
  const long long sites = gr.sites;
  const float dt = L.dt;
  float* __restrict__ out = static_cast<float*>(L.out);
  const int i0 = g * DPT;
  const int oct0 = __float_as_int(t.au[i0].w);
  const bool yneg = oct0 & 2;
  const int zs = (oct0 & 4) ? 1 : 0;
  const int row_own = yneg ? 0 : 1, row_up = yneg ? 1 : 0;
  constexpr int nunits = 2;

  for (int i = g * 32 + lane; i < G * DPT; i += G * 32) {
    const float4 au = t.au[i], nw = t.nw[i];
    const int oct = __float_as_int(au.w);
    const float azw = (oct & 4) ? 1.f - au.z : au.z;
    DirConstM d;
    d.s0 = make_float4(au.x, au.x, au.y, au.y);
    d.s1 = make_float4(azw, azw, nw.x, nw.x);
    d.s2 = make_float4(nw.y, nw.y, nw.z, nw.z);
    d.s3 = make_float4(dt * nw.w, dt * nw.w, 0.f, 0.f);
    d.sh = (oct & 1) ? 1 : -1;
    d.inert = oct & 8;
    d.pad0 = d.pad1 = 0;
    dirs[i] = d;
  }
  if (lane == 0)
    for (int r = 0; r < R; ++r) mbar_init(smem_u32(&mbar[g * R + r]), 1);
  if (g == 0 && lane == 0) *abort_flag = 0;
  // fields of item (tile tix, item mm) into fbuf[b]: invalid sites read
  // site 0, absent fields take their scalar (velocity 0)
  auto stage = [&](int tix, int mm, int b) {
    const TileGeom tq = tile_geom(tix, nxb, ny, nz, L.nzc);
    const int zq = tq.zbeg - 1 + mm;
    const bool zokq = zq >= tq.zbeg && zq < tq.zbeg + tq.zlen;
    float* dst = fbuf + b * 6 * 64;
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int f = 2 * lane + h, x = tq.x0 + f;
      const long long st = zokq && x < nx ? ((long long)zq * ny + tq.y) * nx + x : 0;
      auto put = [&](int c, const float* p, long long off, float sc) {
        if (p) cp_async4(dst + c * 64 + f, p + off);
        else dst[c * 64 + f] = sc;
      };
      put(0, mc.v, st, 0.f);
      put(1, mc.v, sites + st, 0.f);
      put(2, mc.v, 2 * sites + st, 0.f);
      put(3, mc.kta, st, mc.kta_s);
      put(4, mc.kt0, st, mc.kt0_s);
      put(5, mc.etat, st, mc.etat_s);
    }
  };
  if (g == G - 1 && (int)blockIdx.x < ntiles) {
    stage(blockIdx.x, 0, 0);
    cp_async_wait_all();
  }
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();
  unsigned inert_mask = 0;
#pragma unroll
  for (int k = 0; k < DPT; ++k) inert_mask |= dirs[i0 + k].inert ? 1u << k : 0u;

  float* my_ring = ring + (size_t)g * R * SLOT;
  bool alive = true;
  int issued = 0, waited = 0;
  int is_t = blockIdx.x, is_m = 0, is_M = 0, is_x0 = 0, is_yp = 0, is_zp = 0;
  auto issue_seek = [&]() {
    if (is_t < ntiles) {
      const TileGeom tg = tile_geom(is_t, nxb, ny, nz, L.nzc);
      is_M = tile_items<ZC>(tg.zlen);
      is_x0 = tg.x0;
      is_yp = yneg ? tg.y + 1 : tg.y;
      is_zp = tg.zbeg + zs;
    }
  };
  issue_seek();
  auto issue = [&]() -> bool {
    if (is_t >= ntiles || !alive) return false;
    const int slot = issued % R;
    __syncwarp();
    if (lane == 0) {
      const uint32_t bar = smem_u32(&mbar[g * R + slot]);
      fence_proxy_async();
      mbar_arrive_tx(bar, BOXX * DPT * 2 * ZC * 4);
      tma_load_4d(smem_u32(my_ring + (size_t)slot * SLOT), &tmap, is_x0, i0, is_yp,
                  is_zp + is_m * ZC, bar);
    }
    ++issued;
    if (++is_m == is_M) {
      is_m = 0;
      is_t += gridDim.x;
      issue_seek();
    }
    return true;
  };
  auto wait_item = [&](int q) -> bool {
    if (!alive || *abort_flag) {
      alive = false;
      return false;
    }
    if (!mbar_wait(smem_u32(&mbar[g * R + q % R]), (uint32_t)((q / R) & 1), L.err)) {
      *abort_flag = 1;
      alive = false;
      return false;
    }
    waited = q + 1;
    return true;
  };
  const int wc = 2 + 2 * lane;
  while (issued < R - 1 && issue()) {
  }

  float2 carry[DPT];
#pragma unroll
  for (int k = 0; k < DPT; ++k) carry[k] = make_float2(0.f, 0.f);
  float bud_a = 0.f, bud_b = 0.f;
  double bud_da = 0.0, bud_db = 0.0;
  const float2 one2 = make_float2(1.f, 1.f);
  int q = 0;
  for (int ti = blockIdx.x; ti < ntiles; ti += gridDim.x) {
    const TileGeom tg = tile_geom(ti, nxb, ny, nz, L.nzc);
    const int x0 = tg.x0, y = tg.y, zbeg = tg.zbeg, zend = tg.zbeg + tg.zlen;
    const int M = tile_items<ZC>(tg.zlen);
    const int xa = x0 + 2 * lane;
    const bool in0 = xa < nx, in1 = xa + 1 < nx;
    const bool gx_lo = gr.periodic[0] && (xa == nx - 1 || xa + 1 == nx - 1);
    const bool gx_hi = gr.periodic[0] && xa == 0;
    const bool lo_from_y = xa + 1 == nx - 1;
    // fast path (every lane a full pair, so no lane holds both x = 0 and
    // x = nx - 1): the lane's one ghost-column store as offset, value select
    // and predicate
    const bool gx_any = gx_lo || gx_hi;
    const int gx_off = gx_lo ? GL - 1 - (xa + GL) : nx + GL - (xa + GL);
    const bool gx_y = gx_lo && lo_from_y;
    const bool y_face = gr.periodic[1] && (y == 0 || y == ny - 1);
    float* const orow = out + (long long)i0 * gr.si + (long long)(y + 1) * gr.sy + xa + GL;
    for (int m = 0; m < M; ++m, ++q) {
      const int z = zbeg - 1 + m;  // output plane of this item
      const bool zok = z >= zbeg && z < zend;
      // the next item's fields go in while this one is computed
      if (g == G - 1) {
        int tn = ti, mn = m + 1;
        if (mn == M) {
          tn = ti + gridDim.x;
          mn = 0;
        }
        if (tn < ntiles) stage(tn, mn, (q + 1) & 1);
      }
      const float* fb = fbuf + (q & 1) * 6 * 64;
      // per-site fields of the lane's pair: v, W, c_A = dt W (kt_a + kt_0), eta_t
      float2 vx, vy, vz, W, cA, et;
      {
        const float2* f2 = reinterpret_cast<const float2*>(fb) + lane;
        vx = f2[0];
        vy = f2[32];
        vz = f2[64];
        const float2 ka = f2[96], k0 = f2[128];
        et = f2[160];
        const float2 v2 = f2fma(vz, vz, f2fma(vy, vy, f2mul(vx, vx)));
        W = make_float2(rsqrtf(1.f - v2.x), rsqrtf(1.f - v2.y));
        cA = f2mul(f2mul(make_float2(dt, dt), W), make_float2(ka.x + k0.x, ka.y + k0.y));
      }
      // beta_i, A_i, g_i of direction constants d for the lane's pair
      auto coll = [&](const DirConstM& d, float2& beta, float2& A, float2& gg) {
        const float4 s1 = d.s1, s2 = d.s2, s3 = d.s3;
        const float2 vn = f2fma(vz, make_float2(s2.z, s2.w),
                                f2fma(vy, make_float2(s2.x, s2.y), f2mul(vx, make_float2(s1.z, s1.w))));
        beta = f2sub(one2, vn);
        A = f2rcp(f2fma(cA, beta, one2));
        const float2 iw = f2rcp(f2mul(W, beta));
        gg = f2mul(f2mul(A, make_float2(s3.x, s3.y)), f2mul(iw, f2mul(iw, iw)));
      };
      while (issued < q + R && issue()) {
      }
      wait_item(q);
      float* slot = my_ring + (size_t)(q % R) * SLOT;
      const float* own = slot + row_own * DPT * BOXX + wc;
      const float* up = slot + row_up * DPT * BOXX + wc;
      float2 Is[DPT];
      float2 aS = make_float2(0.f, 0.f), aX = aS, aY = aS, aA = aS, aG = aS;
#pragma unroll
      for (int k = 0; k < DPT; ++k) {
        const DirConstM& d = dirs[i0 + k];
        const float4 s0 = d.s0, s1 = d.s1;
        const float2 ax = make_float2(s0.x, s0.y), ay = make_float2(s0.z, s0.w);
        const float2 az = make_float2(s1.x, s1.y);
        const int off = k * BOXX;
        const float2 P0 = *reinterpret_cast<const float2*>(own + off);
        const float2 P1 = *reinterpret_cast<const float2*>(up + off);
        // the x-upwind pair shares one value with the lane's own pair; one
        // 4-byte load completes it (the x sign is uniform over the warp)
        float2 S0, S1;
        if (d.sh > 0) {
          S0 = make_float2(P0.y, own[off + 2]);
          S1 = make_float2(P1.y, up[off + 2]);
        } else {
          S0 = make_float2(own[off - 1], P0.x);
          S1 = make_float2(up[off - 1], P1.x);
        }
        const float2 X0 = f2fma(ax, f2sub(S0, P0), P0);
        const float2 X1 = f2fma(ax, f2sub(S1, P1), P1);
        const float2 Bn = f2fma(ay, f2sub(X1, X0), X0);
        const float2 r = f2fma(az, f2sub(carry[k], Bn), Bn);
        carry[k] = Bn;
        Is[k] = r;
        float2 beta, A, gg;
        coll(d, beta, A, gg);
        const float2 ai = f2mul(A, r);
        const float2 b2 = f2mul(beta, beta);
        aS = f2add(aS, r);
        aX = f2fma(b2, f2fma(gg, et, ai), aX);
        aY = f2fma(b2, gg, aY);
        aA = f2add(aA, ai);
        aG = f2add(aG, gg);
      }
      __syncwarp();
      {
        float2* p = reinterpret_cast<float2*>(slot) + lane;
        p[0] = aS;
        p[32] = aX;
        p[64] = aY;
        p[96] = aA;
        p[128] = aG;
      }
      // the next item's fields have landed before the barrier that publishes them
      if (g == G - 1) cp_async_wait_all();
      __syncthreads();
      // coefficient units: src = eta_t + kt_0 J per site, J = W^2 X / (1 - kt_0 W^2 Y)
      for (int u = g; u < nunits; u += G) {
        const int f = (u << 5) + lane;
        const int x = x0 + f;
        const bool v = zok && x < nx;
        const long long st = v ? ((long long)z * ny + y) * nx + x : 0;
        (void)st;
        const float ux = fb[f], uy = fb[64 + f], uz = fb[128 + f];
        const float kt0 = fb[256 + f], etat = fb[320 + f];
        const int s = q % R;
        float S = 0.f, X = 0.f, Y = 0.f, SA = 0.f, SG = 0.f;
        for (int qq = 0; qq < G; ++qq) {
          const float* p = ring + ((size_t)qq * R + s) * SLOT + f;
          S += p[0];
          X += p[64];
          Y += p[128];
          SA += p[192];
          SG += p[256];
        }
        const float W2 = __fdividef(1.f, 1.f - fmaf(uz, uz, fmaf(uy, uy, ux * ux)));
        const float J = __fdividef(W2 * X, 1.f - kt0 * W2 * Y);
        const float src = fmaf(kt0, J, etat);
        srcs[f] = src;
        if (v) {
          bud_a += S;
          bud_b += fmaf(SG, src, SA);
        }
      }
      __syncthreads();
      if (L.budget_partials && g < nunits) {
        bud_da += (double)bud_a;
        bud_db += (double)bud_b;
        bud_a = bud_b = 0.f;
      }
      const float2 src = reinterpret_cast<const float2*>(srcs)[lane];
      const bool zface = gr.periodic[2] && (z == 0 || z == nz - 1);
      const bool fast = __all_sync(0xffffffffu, in0 && in1) && zok &&
                        !(y_face && ny == 1) && !(zface && nz == 1);
      const bool xghost = __any_sync(0xffffffffu, gx_lo || gx_hi);
      const int yface_rows = (y == ny - 1 ? 0 : ny + 1) - (y + 1);
      if (alive && fast) {
        float* base = orow + (long long)(z + 1) * gr.sz;
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
          if (inert_mask >> k & 1u) continue;
          float2 beta, A, gg;
          coll(dirs[i0 + k], beta, A, gg);
          const float2 o = f2fma(gg, src, f2mul(A, Is[k]));
          float* dst = base + (long long)k * gr.si;
          if constexpr (!PER) {
            *reinterpret_cast<float2*>(dst) = o;
          } else {
            auto put = [&](float* dd) {
              *reinterpret_cast<float2*>(dd) = o;
              if (xghost && gx_any) dd[gx_off] = gx_y ? o.y : o.x;  // one predicated store
            };
            put(dst);
            if (y_face) put(dst + (long long)yface_rows * gr.sy);
            if (zface) {
              const long long zd = (long long)((z == nz - 1 ? 0 : nz + 1) - (z + 1)) * gr.sz;
              put(dst + zd);
              if (y_face) put(dst + zd + (long long)yface_rows * gr.sy);
            }
          }
        }
      } else if (alive && in0 && zok) {
        // partial tile or an extent of 1 on a periodic axis: every image
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
          if (inert_mask >> k & 1u) continue;
          float2 beta, A, gg;
          coll(dirs[i0 + k], beta, A, gg);
          const float2 o = f2fma(gg, src, f2mul(A, Is[k]));
          store_pop(out, gr, i0 + k, z, y, xa, o.x);
          if (in1) store_pop(out, gr, i0 + k, z, y, xa + 1, o.y);
        }
      }
    }
  }
  for (int qq = waited; qq < issued; ++qq)
    mbar_wait(smem_u32(&mbar[g * R + qq % R]), (uint32_t)((qq / R) & 1), L.err);
  if (L.budget_partials) {
    for (int s = 16; s > 0; s >>= 1) {
      bud_da += __shfl_xor_sync(0xffffffffu, bud_da, s);
      bud_db += __shfl_xor_sync(0xffffffffu, bud_db, s);
    }
    if (lane == 0 && g < nunits) {
      bsum[2 * g] = bud_da;
      bsum[2 * g + 1] = bud_db;
    }
    __syncthreads();
    if (g == 0 && lane == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < min(G, nunits); ++w) {
        a += bsum[2 * w];
        b += bsum[2 * w + 1];
      }
      atomicAdd(L.budget_partials + 2 * blockIdx.x, a);
      atomicAdd(L.budget_partials + 2 * blockIdx.x + 1, b);
    }
  }
}

template <int DPT, int R>
size_t smem_moving(int G) {
  return sizeof(float) * ((size_t)G * R * slot_floats<DPT, 1>() + 64 + 2 * 6 * 64) +
         sizeof(DirConstM) * (size_t)G * DPT + 8 * (size_t)G * R + sizeof(double) * 4 + 16;
}

template <bool PER, int DPT, int R, int MAXT, int REGS>
cudaError_t set_attr_moving() {
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && (attr_set >> dev & 1ull)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(k_step_moving_tma<PER, DPT, R, MAXT, REGS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024 - 1024);
  if (e == cudaSuccess && dev < 64) attr_set |= 1ull << dev;
  return e;
}

template <int DPT, int R, int MAXT, int REGS>
cudaError_t occupancy_moving_t(int G, int* per_sm) {
  int a = 0, b = 0;
  cudaError_t e = set_attr_moving<false, DPT, R, MAXT, REGS>();
  if (e == cudaSuccess) e = set_attr_moving<true, DPT, R, MAXT, REGS>();
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &a, k_step_moving_tma<false, DPT, R, MAXT, REGS>, 32 * G, smem_moving<DPT, R>(G));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &b, k_step_moving_tma<true, DPT, R, MAXT, REGS>, 32 * G, smem_moving<DPT, R>(G));
  *per_sm = std::min(a, b);
  return e;
}

template <int DPT, int R, int MAXT, int REGS>
cudaError_t launch_moving_t(const StepLaunch& L, const MovingCoef& c, const DirTable& t,
                            cudaStream_t s, int* nblocks) {
  const int G = L.N / DPT;
  if (!L.tmap_in || G < 1 || G * DPT != L.N || 32 * G > MAXT || L.nzc < 1 || L.nzc > L.g.nz ||
      L.ctas < 1)
    return cudaErrorInvalidValue;
  if (L.budget_partials && L.ctas > L.partials_cap) return cudaErrorInvalidValue;
  if (nblocks) *nblocks = L.ctas;
  const size_t smem = smem_moving<DPT, R>(G);
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  const bool per = L.g.periodic[0] || L.g.periodic[1] || L.g.periodic[2];
  const cudaError_t e = per ? set_attr_moving<true, DPT, R, MAXT, REGS>()
                            : set_attr_moving<false, DPT, R, MAXT, REGS>();
  if (e != cudaSuccess) return e;
  if (per)
    k_step_moving_tma<true, DPT, R, MAXT, REGS><<<L.ctas, dim3(32, G), smem, s>>>(*L.tmap_in, L, c, t);
  else
    k_step_moving_tma<false, DPT, R, MAXT, REGS><<<L.ctas, dim3(32, G), smem, s>>>(*L.tmap_in, L, c, t);
  return cudaGetLastError();
}

constexpr int kRingM = 2;

// Tile plans of the moving kernel (directions per warp, thread cap,
// registers); one plane per batch.
#define LBRT_MOVING_PLANS(X) \
  X(5, 320, 96)              \
  X(11, 512, 128)            \
  X(10, 544, 96)

}  // namespace

#define LBRT_MROW(D, T, B) {D, 1, T},
const int kTilePlansMoving[][3] = {LBRT_MOVING_PLANS(LBRT_MROW)};
#undef LBRT_MROW
const int kNumTilePlansMoving = sizeof(kTilePlansMoving) / sizeof(kTilePlansMoving[0]);

size_t step_tile_smem_moving(int dpt, int warps) {
#define LBRT_MS(D, T, B) \
  if (dpt == D) return smem_moving<D, kRingM>(warps);
  LBRT_MOVING_PLANS(LBRT_MS)
#undef LBRT_MS
  return (size_t)-1;
}

cudaError_t occupancy_tma_moving(int dpt, int G, int* per_sm) {
#define LBRT_MO(D, T, B) \
  if (dpt == D) return occupancy_moving_t<D, kRingM, T, B>(G, per_sm);
  LBRT_MOVING_PLANS(LBRT_MO)
#undef LBRT_MO
  return cudaErrorInvalidValue;
}

cudaError_t launch_tma_moving(const StepLaunch& L, const MovingCoef& c, const DirTable& t,
                              cudaStream_t s, int* nblocks) {
#define LBRT_ML(D, T, B) \
  if (L.dpt == D && L.zc == 1) return launch_moving_t<D, kRingM, T, B>(L, c, t, s, nblocks);
  LBRT_MOVING_PLANS(LBRT_ML)
#undef LBRT_ML
  return cudaErrorInvalidValue;
}

}  // namespace lbrt
