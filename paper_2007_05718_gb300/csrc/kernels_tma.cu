// Fused stream + collide step for a static fluid, float32 populations, fed
// by TMA tensor tiles.  Weih et al. 2020: Sec. 3.3, Eqs. (interp),
// (rte_implicit), (collision-step).
//
// Work decomposition.  A CTA owns 64 consecutive x sites of one row y and a
// chunk of planes in z; each lane owns an x-pair (2 sites, packed FFMA2
// arithmetic).  Warp g owns the DPT directions g DPT .. g DPT + DPT - 1 of the
// library's internal direction order, in which directions are grouped by
// (sgn n^y, sgn n^z) and every group is padded to a multiple of DPT with inert
// zero-weight directions; so all directions of a warp pull from the same
// upwind row and plane.  The chunk is processed in batches of ZC planes.
//
// Data movement.  Per batch a warp needs, for each of its directions and
// each of the ZC planes, the own row y and the upwind row y - sgn(n^y) over
// the columns x0 - 2 .. x0 + 65.  In the padded layout [z][y][dir][x] these
// form ONE box of 68 x DPT x 2 x ZC floats (the ghost layer supplies
// periodic images and vacuum zeros), fetched by a single TMA load issued by
// lane 0; large boxes keep the copy engine near full bandwidth.  Each warp
// double-buffers its boxes (the next batch is in flight while the current
// one is computed).  Waits are bounded: a wait that gives up sets the device
// error word and the CTA runs to its end without further compute.
//
// Arithmetic per direction and plane: the bilinear value of the two rows
// (x then y), a lerp in z against the plane carried in a register from the
// previous plane (Eq. interp factorised), I* kept in registers and the
// partial (E*, F*) accumulated; after the batch, one CTA barrier exchanges
// the G partial moments, every warp forms the collision scalars of its own
// lanes' sites, and I_i^{n+1} = alpha I*_i + w_i (c0 + n_i . c1) is stored as
// float2 (plus ghost mirrors at periodic faces).
#include <algorithm>

#include "lb_rt_internal.h"

#include <cudaTypedefs.h>

namespace lbrt {

namespace {

// ---- packed float32 x 2 arithmetic (FFMA2 / FADD2 / FMUL2 builtins) -------
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
// t a + (1 - t) b as two fused multiply-adds, with nt = -t precomputed
__device__ __forceinline__ float2 f2lerp(float2 t, float2 nt, float2 a, float2 b) {
  return __ffma2_rn(t, a, __ffma2_rn(nt, b, b));
}

// ---- mbarrier and TMA ------------------------------------------------------
__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive_tx(uint32_t bar, uint32_t bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ void tma_load_4d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, int c3, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.4d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4, %5}], [%6];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(c3), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

constexpr int BOXX = 68;                          // columns x0 - 2 .. x0 + 65
constexpr long long WAIT_CYCLES = 4000000000LL;   // ~2 s at 2 GHz: longer is a fault

// Bounded wait on an mbarrier phase.  Returns false (and sets the error
// word) when the phase has not completed within WAIT_CYCLES SM cycles.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, unsigned* err) {
  if (mbar_try(bar, parity)) return true;
  const long long t0 = clock64();
  int spins = 0;
  while (!mbar_try(bar, parity)) {
    if ((++spins & 63) == 0 && clock64() - t0 > WAIT_CYCLES) {
      atomicOr(err, 1u);
      return false;
    }
  }
  return true;
}

__device__ __forceinline__ float fld(const float* __restrict__ p, float s, long long i) {
  return p ? __ldg(p + i) : s;
}

struct Coef {
  float alpha, c0, c1x, c1y, c1z, Enew;
};

// Site scalars of the static collision such that
//   I_i^{n+1} = alpha I*_i + w_i (c0 + n_i . c1).
//   implicit exact (Eq. rte_implicit, isotropic table), A = 1/(1 + dt (k0 + ka)):
//     E = (E* + dt eta) / (1 + dt ka),  F = F* / (1 + dt (ka + k0) - dt k0 lam / d),
//     alpha = A, c0 = A dt (eta + k0 E) = E - A E*, c1 = A dt k0 lam F.
//     c0 is evaluated in the residual form E - A E*, which keeps
//     sum_i I_i^{n+1} = E free of a systematic float32 bias in A (pure
//     scattering: E = E* exactly, so energy is conserved to rounding);
//   explicit (Eq. collision-step): alpha = 1 - dt (k0 + ka),
//     c0 = dt (k0 E* + eta) = E_new - alpha E* with E_new = E* + dt (eta - ka E*),
//     c1 = dt k0 lam F*;
//   Lambda-K (Sec. 3.3): K passes started from (E*, F*); for an isotropic
//     table a pass maps (E, F) -> (A (E* + dt eta + dt k0 E), A (F* + dt k0 lam F / d)),
//     and the output populations are those of pass K, built from the
//     moments of pass K - 1.
__device__ __forceinline__ Coef collide_scalars(int mode, int iters, float dt, float inv_d,
                                                float ka, float k0, float lam, float eta,
                                                float Es, float Fx, float Fy, float Fz) {
  Coef c;
  if (mode == LB_RT_EXPLICIT) {
    c.alpha = 1.f - dt * (k0 + ka);
    c.Enew = fmaf(dt, eta - ka * Es, Es);
    c.c0 = fmaf(-c.alpha, Es, c.Enew);
    const float g = dt * k0 * lam;
    c.c1x = g * Fx; c.c1y = g * Fy; c.c1z = g * Fz;
    return c;
  }
  const float A = 1.f / (1.f + dt * (k0 + ka));
  float gx, gy, gz;
  if (mode == LB_RT_LAMBDA_K) {
    float E = Es;
    gx = Fx; gy = Fy; gz = Fz;
    const float q = dt * k0 * lam * inv_d;
    for (int m = 1; m < iters; ++m) {
      E = A * (Es + dt * eta + dt * k0 * E);
      gx = A * (Fx + q * gx); gy = A * (Fy + q * gy); gz = A * (Fz + q * gz);
    }
    c.c0 = A * dt * (eta + k0 * E);
    c.Enew = fmaf(A, Es, c.c0);
  } else {
    const float E = (Es + dt * eta) / (1.f + dt * ka);
    const float r = 1.f / (1.f + dt * (ka + k0) - dt * k0 * lam * inv_d);
    gx = Fx * r; gy = Fy * r; gz = Fz * r;
    c.c0 = fmaf(-A, Es, E);
    c.Enew = E;
  }
  c.alpha = A;
  const float g = A * dt * k0 * lam;
  c.c1x = g * gx; c.c1y = g * gy; c.c1z = g * gz;
  return c;
}

template <int DPT, int ZC>
__host__ __device__ constexpr int slot_floats() {
  return ((BOXX * DPT * 2 * ZC * 4 + 127) / 128) * 32;  // 128-byte aligned slots
}

// In-plane bilinear value of the lane's pair from one box row pair: r0 the
// own row, r1 the upwind row (pointers at the window column of the pair),
// upwind column at offset `du` (-1 or +2) from the pair's first site.
__device__ __forceinline__ float2 bilinear(const float* r0, const float* r1, int du, bool xneg,
                                           float2 ax, float2 nax, float2 ay, float2 nay) {
  const float2 v0 = *reinterpret_cast<const float2*>(r0);
  const float2 v1 = *reinterpret_cast<const float2*>(r1);
  const float u0 = r0[du], u1 = r1[du];
  const float2 w0 = xneg ? make_float2(v0.y, u0) : make_float2(u0, v0.x);
  const float2 w1 = xneg ? make_float2(v1.y, u1) : make_float2(u1, v1.x);
  return f2lerp(ay, nay, f2lerp(ax, nax, w1, v1), f2lerp(ax, nax, w0, v0));
}

template <int DPT, int ZC, int R, int MAXT>
__global__ void __launch_bounds__(MAXT, 1)
k_step_f32(const __grid_constant__ CUtensorMap tmap, const StepLaunch L, const StaticCoef cf,
           const DirTable t, int zchunk) {
  constexpr int SLOT = slot_floats<DPT, ZC>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int G = blockDim.y;
  const int lane = threadIdx.x, g = threadIdx.y;
  const Grid& gr = L.g;
  const int nx = gr.nx, ny = gr.ny, nz = gr.nz;
  // shared layout: ring [G][R][SLOT] | part [2][G][ZC][4][32] float2 | mbar [G][R] | abort flag
  float* ring = reinterpret_cast<float*>(smem_raw);
  float2* part2 = reinterpret_cast<float2*>(ring + (size_t)G * R * SLOT);
  unsigned long long* mbar =
      reinterpret_cast<unsigned long long*>(part2 + (size_t)2 * G * ZC * 4 * 32);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(mbar + G * R);

  const int x0 = blockIdx.x * 64;
  const int xa = x0 + 2 * lane;  // the lane's pair (xa, xa + 1)
  const bool in0 = xa < nx, in1 = xa + 1 < nx;
  const int y = blockIdx.y;
  const int zbeg = blockIdx.z * zchunk;
  const int zend = min(zbeg + zchunk, nz);
  const float inv_d = 1.f / (float)gr.dims;
  float* __restrict__ out = static_cast<float*>(L.out);
  const int nbatch = (zend - zbeg + ZC - 1) / ZC;
  const int i0 = g * DPT;
  // the warp's row / plane class (uniform over its directions)
  const int oct0 = __float_as_int(t.au[i0].w);
  const bool yneg = oct0 & 2;
  const int zs = (oct0 & 4) ? 1 : 0;
  const int row_own = yneg ? 0 : 1, row_up = yneg ? 1 : 0;

  if (lane == 0) {
    for (int r = 0; r < R; ++r) mbar_init(smem_u32(&mbar[g * R + r]), 1);
  }
  if (g == 0 && lane == 0) *abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  float* my_ring = ring + (size_t)g * R * SLOT;
  bool alive = true;
  int issued = 0;
  // item q = batch q - 1 (q = 0: the plane below the chunk, for the carries)
  auto issue = [&](int q) {
    if (q > nbatch || !alive) return;
    issued = q + 1;
    __syncwarp();
    if (lane == 0) {
      const int slot = q % R;
      const uint32_t bar = smem_u32(&mbar[g * R + slot]);
      const int zp = (q == 0 ? zbeg - 1 : zbeg + (q - 1) * ZC) + zs + 1;  // padded plane
      const int yp = yneg ? y + 1 : y;                                 // lower row (padded)
      fence_proxy_async();
      mbar_arrive_tx(bar, BOXX * DPT * 2 * ZC * 4);
      tma_load_4d(smem_u32(my_ring + (size_t)slot * SLOT), &tmap, x0, i0, yp, zp, bar);
    }
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
    return true;
  };
  // element (plane j, row r, direction k) of a slot, at the lane's pair
  const int wc = 2 + 2 * lane;  // window column of xa: x - (x0 - 2)
  auto at = [&](const float* slot, int j, int r, int k) {
    return slot + ((j * 2 + r) * DPT + k) * BOXX + wc;
  };

  for (int r = 0; r < R - 1; ++r) issue(r);

  float2 carry[DPT];
  {
    issue(R - 1);
    const bool ok = wait_item(0);
    const float* slot = my_ring;
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      carry[k] = make_float2(0.f, 0.f);
      if (ok) {
        const float4 au = t.au[i0 + k];
        const bool xneg = __float_as_int(au.w) & 1;
        carry[k] = bilinear(at(slot, 0, row_own, k), at(slot, 0, row_up, k), xneg ? 2 : -1, xneg,
                            f2s(au.x), f2s(-au.x), f2s(au.y), f2s(-au.y));
      }
    }
  }

  double bud_a = 0.0, bud_b = 0.0;
  for (int b = 0; b < nbatch; ++b) {
    const int q = b + 1;
    const int zb = zbeg + b * ZC;
    const int nb = min(ZC, zend - zb);
    float2* part = part2 + (size_t)(b & 1) * G * ZC * 4 * 32;
    // the lane's site coefficients, loaded now so that their latency
    // overlaps the stream pass
    float fka[ZC][2], fk0[ZC][2], flam[ZC][2], feta[ZC][2];
#pragma unroll
    for (int j = 0; j < ZC; ++j) {
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool okx = (xa + h < nx) && (j < nb);
        const long long st = okx ? ((long long)(zb + j) * ny + y) * nx + xa + h : 0;
        fka[j][h] = fld(cf.ka, cf.ka_s, st);
        fk0[j][h] = fld(cf.k0, cf.k0_s, st);
        flam[j][h] = fld(cf.lam, cf.lam_s, st);
        feta[j][h] = fld(cf.eta, cf.eta_s, st);
      }
    }
    issue(q + R - 1);
    const bool ok = wait_item(q);
    const float* slot = my_ring + (size_t)(q % R) * SLOT;
    float2 Is[DPT][ZC];
    float2 aE[ZC], aX[ZC], aY[ZC], aZ[ZC];
#pragma unroll
    for (int j = 0; j < ZC; ++j) aE[j] = aX[j] = aY[j] = aZ[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
#pragma unroll
      for (int j = 0; j < ZC; ++j) Is[k][j] = make_float2(0.f, 0.f);
      if (ok) {
        const float4 au = t.au[i0 + k];
        const float4 nw = t.nw[i0 + k];
        const int oct = __float_as_int(au.w);
        const bool xneg = oct & 1;
        const float2 ax = f2s(au.x), ay = f2s(au.y), nax = f2s(-au.x), nay = f2s(-au.y);
        const float azw = zs ? 1.f - au.z : au.z;
        const float2 az = f2s(azw), naz = f2s(-azw);
        const float2 nx2 = f2s(nw.x), ny2 = f2s(nw.y), nz2 = f2s(nw.z);
#pragma unroll
        for (int j = 0; j < ZC; ++j) {
          const float2 Bn = bilinear(at(slot, j, row_own, k), at(slot, j, row_up, k),
                                     xneg ? 2 : -1, xneg, ax, nax, ay, nay);
          // I* = (1 - a_z) B(z) + a_z B(z - sgn n^z): the carried plane is
          // B(z - 1) for sgn = +1 and B(z) for sgn = -1
          const float2 r = f2lerp(az, naz, carry[k], Bn);
          carry[k] = Bn;
          Is[k][j] = r;
          aE[j] = f2add(aE[j], r);
          aX[j] = f2fma(nx2, r, aX[j]);
          aY[j] = f2fma(ny2, r, aY[j]);
          aZ[j] = f2fma(nz2, r, aZ[j]);
        }
      }
    }
#pragma unroll
    for (int j = 0; j < ZC; ++j) {
      float2* p = part + (((size_t)g * ZC + j) * 4) * 32 + lane;
      p[0] = aE[j];
      p[32] = aX[j];
      p[64] = aY[j];
      p[96] = aZ[j];
    }
    __syncthreads();
    // every warp sums the G partials of its own lanes' sites and forms the
    // collision scalars itself (no second barrier; the partials are double
    // buffered across batches)
    float2 al[ZC], c0[ZC], c1x[ZC], c1y[ZC], c1z[ZC];
    float ea = 0.f, eb = 0.f;  // this batch's budget terms, folded into FP64 below
#pragma unroll
    for (int j = 0; j < ZC; ++j) {
      float2 E = make_float2(0.f, 0.f), Fx = E, Fy = E, Fz = E;
      for (int qq = 0; qq < G; ++qq) {
        const float2* p = part + (((size_t)qq * ZC + j) * 4) * 32 + lane;
        E = f2add(E, p[0]);
        Fx = f2add(Fx, p[32]);
        Fy = f2add(Fy, p[64]);
        Fz = f2add(Fz, p[96]);
      }
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float Es = h ? E.y : E.x;
        const Coef cc = collide_scalars(L.collision, L.lambda_iters, L.dt, inv_d, fka[j][h],
                                        fk0[j][h], flam[j][h], feta[j][h], Es,
                                        h ? Fx.y : Fx.x, h ? Fy.y : Fy.x, h ? Fz.y : Fz.x);
        (h ? al[j].y : al[j].x) = cc.alpha;
        (h ? c0[j].y : c0[j].x) = cc.c0;
        (h ? c1x[j].y : c1x[j].x) = cc.c1x;
        (h ? c1y[j].y : c1y[j].x) = cc.c1y;
        (h ? c1z[j].y : c1z[j].x) = cc.c1z;
        if (j < nb && xa + h < nx) {
          ea += Es;
          eb += cc.Enew;
        }
      }
    }
    if (L.budget_partials && g == 0) {
      bud_a += (double)ea;
      bud_b += (double)eb;
    }
    if (alive && in0) {
      // x ghost columns this lane mirrors into (periodic x): column GL - 1
      // holds x = nx - 1, column nx + GL holds x = 0
      const bool gx_lo = gr.periodic[0] && (xa == nx - 1 || xa + 1 == nx - 1);
      const bool gx_hi = gr.periodic[0] && xa == 0;
      const bool lo_from_y = xa + 1 == nx - 1;
      const bool y_face = gr.periodic[1] && (y == 0 || y == ny - 1);
#pragma unroll
      for (int k = 0; k < DPT; ++k) {
        const float4 nw = t.nw[i0 + k];
        if (__float_as_int(t.au[i0 + k].w) & 8) continue;  // inert padding direction
        const float2 nx2 = f2s(nw.x), ny2 = f2s(nw.y), nz2 = f2s(nw.z), w2 = f2s(nw.w);
#pragma unroll
        for (int j = 0; j < ZC; ++j) {
          if (j < nb) {
            const int z = zb + j;
            const float2 eq = f2fma(nz2, c1z[j], f2fma(ny2, c1y[j], f2fma(nx2, c1x[j], c0[j])));
            const float2 o = f2fma(al[j], Is[k][j], f2mul(w2, eq));
            const float vlo = lo_from_y ? o.y : o.x;
            const bool z_face = gr.periodic[2] && (z == 0 || z == nz - 1);
            if (!(y_face || z_face)) {
              float* base = out + (long long)(i0 + k) * gr.si + (long long)(z + 1) * gr.sz +
                            (long long)(y + 1) * gr.sy;
              if (in1) *reinterpret_cast<float2*>(base + xa + GL) = o;
              else base[xa + GL] = o.x;
              if (gx_lo) base[GL - 1] = vlo;
              if (gx_hi) base[nx + GL] = o.x;
            } else {
              // a row or plane on a periodic face: every (row, plane) image
              const int rows[3] = {y + 1, (gr.periodic[1] && y == ny - 1) ? 0 : -1,
                                   (gr.periodic[1] && y == 0) ? ny + 1 : -1};
              const int planes[3] = {z + 1, (gr.periodic[2] && z == nz - 1) ? 0 : -1,
                                     (gr.periodic[2] && z == 0) ? nz + 1 : -1};
#pragma unroll 1
              for (int cmb = 0; cmb < 9; ++cmb) {
                const int rr = rows[cmb % 3], pp = planes[cmb / 3];
                if (rr < 0 || pp < 0) continue;
                float* base = out + (long long)(i0 + k) * gr.si + (long long)pp * gr.sz +
                              (long long)rr * gr.sy;
                base[xa + GL] = o.x;
                if (in1) base[xa + GL + 1] = o.y;
                if (gx_lo) base[GL - 1] = vlo;
                if (gx_hi) base[nx + GL] = o.x;
              }
            }
          }
        }
      }
    }
  }
  // every issued copy must land before the CTA's shared memory is released
  for (int qq = nbatch + 1; qq < issued; ++qq)
    mbar_wait(smem_u32(&mbar[g * R + qq % R]), (uint32_t)((qq / R) & 1), L.err);
  if (!alive) {
    for (int qq = 0; qq < issued; ++qq)
      mbar_wait(smem_u32(&mbar[g * R + qq % R]), (uint32_t)((qq / R) & 1), L.err);
  }
  if (L.budget_partials) {
    for (int s = 16; s > 0; s >>= 1) {
      bud_a += __shfl_xor_sync(0xffffffffu, bud_a, s);
      bud_b += __shfl_xor_sync(0xffffffffu, bud_b, s);
    }
    if (lane == 0) {
      const long long blk =
          ((long long)blockIdx.z * gridDim.y + blockIdx.y) * gridDim.x + blockIdx.x;
      atomicAdd(L.budget_partials + 2 * blk, bud_a);
      atomicAdd(L.budget_partials + 2 * blk + 1, bud_b);
    }
  }
}

template <int DPT, int ZC, int R>
size_t step_smem(int G) {
  return sizeof(float) * (size_t)G * R * slot_floats<DPT, ZC>() +
         sizeof(float2) * 32 * ((size_t)2 * G * ZC * 4) + 8 * (size_t)G * R + 16;
}

template <int DPT, int ZC, int R, int MAXT>
cudaError_t launch_f32(const StepLaunch& L, const StaticCoef& c, const DirTable& t, int zchunk,
                       cudaStream_t s, int* nblocks) {
  const int G = L.N / DPT;  // internal (padded) direction count / directions per warp
  if (!L.tmap_in || G < 1 || G * DPT != L.N || 32 * G > MAXT) return cudaErrorInvalidValue;
  dim3 block(32, G);
  dim3 grid((L.g.nx + 63) / 64, L.g.ny, (L.g.nz + zchunk - 1) / zchunk);
  const long long nb_ = (long long)grid.x * grid.y * grid.z;
  if (L.budget_partials && nb_ > L.partials_cap) return cudaErrorInvalidValue;
  if (nblocks) *nblocks = (int)nb_;
  const size_t smem = step_smem<DPT, ZC, R>(G);
  if (smem > 227 * 1024) return cudaErrorInvalidValue;
  // the opt-in shared-memory size is a per-device function attribute
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !(attr_set >> dev & 1ull)) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_step_f32<DPT, ZC, R, MAXT>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    attr_set |= 1ull << dev;
  }
  k_step_f32<DPT, ZC, R, MAXT><<<grid, block, smem, s>>>(*L.tmap_in, L, c, t, zchunk);
  return cudaGetLastError();
}

constexpr int kRing = 2;

}  // namespace

// Compiled tile plans (directions per warp, planes per batch, thread cap of
// the launch bounds), in order of preference for the host's planner, which
// also checks the shared-memory need with step_tile_smem().
const int kTilePlans[][3] = {{5, 2, 512}, {10, 1, 640}, {8, 2, 512}, {4, 2, 512}, {4, 1, 768}};
const int kNumTilePlans = 5;

size_t step_tile_smem(int dpt, int zc, int warps) {
  if (dpt == 5 && zc == 2) return step_smem<5, 2, kRing>(warps);
  if (dpt == 10 && zc == 1) return step_smem<10, 1, kRing>(warps);
  if (dpt == 8 && zc == 2) return step_smem<8, 2, kRing>(warps);
  if (dpt == 4 && zc == 2) return step_smem<4, 2, kRing>(warps);
  if (dpt == 4 && zc == 1) return step_smem<4, 1, kRing>(warps);
  return (size_t)-1;
}

cudaError_t launch_tma_static(const StepLaunch& L, const StaticCoef& c, const DirTable& t,
                              int dpt, int zc, cudaStream_t s, int* nblocks) {
  const int zchunk = 32;
  if (dpt == 5 && zc == 2) return launch_f32<5, 2, kRing, 512>(L, c, t, zchunk, s, nblocks);
  if (dpt == 10 && zc == 1) return launch_f32<10, 1, kRing, 640>(L, c, t, zchunk, s, nblocks);
  if (dpt == 8 && zc == 2) return launch_f32<8, 2, kRing, 512>(L, c, t, zchunk, s, nblocks);
  if (dpt == 4 && zc == 2) return launch_f32<4, 2, kRing, 512>(L, c, t, zchunk, s, nblocks);
  if (dpt == 4 && zc == 1) return launch_f32<4, 1, kRing, 768>(L, c, t, zchunk, s, nblocks);
  return cudaErrorInvalidValue;
}

bool make_pop_tensor_map(CUtensorMap* map, const Grid& g, int Ni, void* base, int dpt, int zc,
                         std::string& err) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      err = "cuTensorMapEncodeTiled is not available from the driver";
      return false;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  const cuuint64_t dims[4] = {(cuuint64_t)g.PX, (cuuint64_t)Ni, (cuuint64_t)g.PY,
                              (cuuint64_t)g.PZ};
  const cuuint64_t strides[3] = {(cuuint64_t)g.si * 4, (cuuint64_t)g.sy * 4,
                                 (cuuint64_t)g.sz * 4};
  const cuuint32_t box[4] = {(cuuint32_t)BOXX, (cuuint32_t)dpt, 2, (cuuint32_t)zc};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, base, dims, strides, box,
                            estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

}  // namespace lbrt
