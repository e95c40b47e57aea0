// Device helpers shared by the TMA-fed step kernels (float32 and 16-bit
// storage): packed float32 x 2 arithmetic, mbarrier and TMA wrappers with
// bounded waits, the static collision scalars and the persistent tile
// schedule.  Included by kernels_tma.cu and kernels_tma16.cu only.
#pragma once

#include "lb_rt_internal.h"

namespace lbrt {
namespace tma {

// ---- packed float32 x 2 arithmetic (FFMA2 / FADD2 / FMUL2 builtins) -------
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) { return __ffma2_rn(a, b, c); }
__device__ __forceinline__ float2 f2add(float2 a, float2 b) { return __fadd2_rn(a, b); }
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) { return __fmul2_rn(a, b); }
// a - b as one packed FMA, b (-1) + a (exact up to the single rounding)
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
  return __ffma2_rn(b, make_float2(-1.f, -1.f), a);
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
// One bounded try: the thread may be suspended until the phase completes or
// about 20 microseconds pass (the hint is in nanoseconds), so a waiting warp
// does not take issue slots from the warps that have work.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity) {
  uint32_t ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n"
      " selp.u32 %0, 1, 0, p;\n}\n"
      : "=r"(ok)
      : "r"(bar), "r"(parity), "r"(20000u)
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
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, int c0, int c1,
                                            int c2, uint32_t bar) {
  asm volatile(
      "cp.async.bulk.tensor.3d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
      " [%0], [%1, {%2, %3, %4}], [%5];" ::"r"(dst),
      "l"(reinterpret_cast<uint64_t>(map)), "r"(c0), "r"(c1), "r"(c2), "r"(bar)
      : "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// CTA barrier.  A block that runs one tile plan uses __syncthreads(); a
// block of a launch shared by two plans (kernels_tma16.cu, kernels_tma.cu)
// has idle warps that leave at once, so its barriers are named barriers
// counting the nthreads threads of the plan's warps.
template <bool PART>
__device__ __forceinline__ void cta_sync(int nthreads) {
  if constexpr (PART) {
    asm volatile("bar.sync 1, %0;" ::"r"(nthreads) : "memory");
  } else {
    __syncthreads();
  }
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

// 4-byte global -> shared copy that completes asynchronously (cp.async);
// cp_async_wait_all() waits for all of the thread's outstanding copies
__device__ __forceinline__ void cp_async4(float* sdst, const float* gsrc) {
  asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(smem_u32(sdst)), "l"(gsrc)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.wait_all;" ::: "memory");
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
// The quotients use the fast division (a few ulp): every denominator is at
// least 1 for non-negative opacities and lam <= d.
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
  const float A = __fdividef(1.f, 1.f + dt * (k0 + ka));
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
    const float E = __fdividef(Es + dt * eta, 1.f + dt * ka);
    const float r = __fdividef(1.f, 1.f + dt * (ka + k0) - dt * k0 * lam * inv_d);
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

// Tile schedule of the persistent grid: tile ti covers the 64 columns
// x0 .. x0 + 63 of row y over the planes zbeg .. zbeg + zlen - 1; tiles are
// numbered x-block fastest, then y, then z chunk, and CTA b takes tiles b,
// b + gridDim.x, ...  so that the tiles in flight at one time are
// neighbouring rows whose shared upwind rows meet in L2.  The nz planes are
// split into nzc chunks of near-equal length.
struct TileGeom {
  int x0, y, zbeg, zlen;
};
// rot: the x-blocks of the tile's row are permuted cyclically by rot (the
// same rot for every tile of a row keeps the map a bijection).
__device__ __forceinline__ TileGeom tile_geom(int ti, int nxb, int ny, int nz, int nzc,
                                              int rot = 0) {
  TileGeom tg;
  tg.x0 = ((ti % nxb + rot) % nxb) * 64;
  const int r = ti / nxb;
  tg.y = r % ny;
  const int c = r / ny;
  const int base = nz / nzc, rem = nz % nzc;
  tg.zbeg = c * base + min(c, rem);
  tg.zlen = base + (c < rem ? 1 : 0);
  return tg;
}

// Per tile the kernel walks the planes B(zbeg - 1) .. B(zbeg + zlen - 1) of
// the in-plane (bilinear) values, ZC planes per item; item m, plane j yields
// the output plane z = zbeg - 1 + m ZC + j (for both signs of n^z, with the
// box shifted by one plane for sgn n^z = -1), which is stored when it lies in
// the tile; the first plane of a tile only seeds the carried value.
// Rotation of the x-blocks for tile ti (problem-relative) of a persistent
// grid of ncta CTAs.  When ncta is a multiple of the x-blocks per row, CTA b
// would keep one x-block for the whole step; with a periodic x axis the CTAs
// of the first and last x-block also write the ghost columns and fall
// behind.  Rotating the x-blocks of every row by the round ti / ncta makes
// every CTA walk all x-blocks, while the tiles of one round (and so the
// neighbouring rows in flight together) stay the same.  A row never spans
// two rounds because ncta is a multiple of nxb.
__device__ __forceinline__ int tile_rot(int ti, int nxb, int ncta, bool periodic_x) {
  return (periodic_x && nxb > 1 && ncta % nxb == 0) ? ti / ncta : 0;
}

template <int ZC>
__device__ __forceinline__ int tile_items(int zlen) {
  return (zlen + 1 + ZC - 1) / ZC;
}


}  // namespace tma
}  // namespace lbrt
