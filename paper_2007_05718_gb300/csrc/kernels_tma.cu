// Fused stream + collide step for a static fluid, float32 populations, fed
// by TMA tensor tiles.  Weih et al. 2020: Sec. 3.3, Eqs. (interp),
// (rte_implicit), (collision-step).
//
// Work decomposition.  A CTA owns 64 consecutive x sites of one row y and a
// chunk of planes in z; each lane owns an x-pair (2 sites, packed f32x2
// arithmetic).  The G warps split the N directions (DPT each) and the chunk
// is processed in batches of ZC planes.
//
// Data movement.  For every (direction, batch) item a warp needs, per plane,
// the own row y and the upwind row y - sgn(n^y) over the columns
// x0 - 2 .. x0 + 65.  In the padded population layout these are one box of
// 68 x 2 x ZC floats (the ghost layer supplies periodic images and vacuum
// zeros), fetched by a single cp.async.bulk.tensor.3d issued by lane 0 with
// completion counted on an mbarrier.  Each warp keeps a ring of R slots and
// fetches R - 1 items ahead, so later directions (and the next batch,
// across the CTA barriers) are in flight while the current one is computed.
// Waits are bounded: a wait that gives up sets the device error word and the
// CTA runs to its end without further compute.
//
// Arithmetic per item and plane: the bilinear value of the two rows (x then
// y), a lerp in z against the plane carried in a register from the previous
// plane (Eq. interp factorised), I* staged in shared memory and the partial
// (E*, F*) accumulated; after the batch the G partials give the site
// scalars of the collision and I_i^{n+1} = alpha I*_i + w_i (c0 + n_i . c1) is
// stored as float2 (plus ghost mirrors at periodic faces).
#include "lb_rt_internal.h"

#include <cudaTypedefs.h>

namespace lbrt {

namespace {

// ---- packed float32 x 2 arithmetic --------------------------------------
__device__ __forceinline__ unsigned long long pk2(float2 a) {
  unsigned long long r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(a.x), "f"(a.y));
  return r;
}
__device__ __forceinline__ float2 upk2(unsigned long long r) {
  float2 a;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(a.x), "=f"(a.y) : "l"(r));
  return a;
}
__device__ __forceinline__ float2 f2fma(float2 a, float2 b, float2 c) {
  unsigned long long d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)), "l"(pk2(c)));
  return upk2(d);
}
__device__ __forceinline__ float2 f2sub(float2 a, float2 b) {
  unsigned long long d;
  asm("sub.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ float2 f2add(float2 a, float2 b) {
  unsigned long long d;
  asm("add.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ float2 f2mul(float2 a, float2 b) {
  unsigned long long d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(pk2(a)), "l"(pk2(b)));
  return upk2(d);
}
__device__ __forceinline__ float2 f2s(float a) { return make_float2(a, a); }
// weight t on a, 1 - t on b
__device__ __forceinline__ float2 f2lerp(float2 t, float2 a, float2 b) {
  return f2fma(t, f2sub(a, b), b);
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

constexpr int BOXX = 68;                       // columns x0 - 2 .. x0 + 65
constexpr long long WAIT_CYCLES = 4000000000LL;  // ~2 s at 2 GHz: longer is a fault

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

template <int ZC>
__host__ __device__ constexpr int slot_floats() {
  return ((BOXX * 2 * ZC * 4 + 127) / 128) * 32;  // 128-byte aligned slots
}

template <int DPT, int ZC, int R>
__global__ void __launch_bounds__(256)
k_tma_static(const __grid_constant__ CUtensorMap tmap, const StepLaunch L, const StaticCoef cf,
             const DirTable t, int zchunk) {
  extern __shared__ __align__(128) unsigned char smem_raw[];
  constexpr int SLOT = slot_floats<ZC>();
  const int G = blockDim.y;
  const int lane = threadIdx.x, g = threadIdx.y;
  const Grid& gr = L.g;
  const int nx = gr.nx, nz = gr.nz;
  const int NP = G * DPT;
  // shared layout: ring [G][R][SLOT] | I* [NP][ZC][32] float2 | part [G][ZC][4][32] float2 |
  //                coef [ZC][5][32] float2 | mbar [G][R] | abort flag
  float* ring = reinterpret_cast<float*>(smem_raw);
  float2* Ist = reinterpret_cast<float2*>(ring + (size_t)G * R * SLOT);
  float2* part = Ist + (size_t)NP * ZC * 32;
  float2* coef = part + (size_t)G * ZC * 4 * 32;
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(coef + (size_t)ZC * 5 * 32);
  int* abort_flag = reinterpret_cast<int*>(mbar + G * R);

  const int x0 = blockIdx.x * 64;
  const int xa = x0 + 2 * lane;       // the lane's pair (xa, xa + 1)
  const bool in0 = xa < nx, in1 = xa + 1 < nx;
  const int y = blockIdx.y;
  const int zbeg = blockIdx.z * zchunk;
  const int zend = min(zbeg + zchunk, nz);
  const float inv_d = 1.f / (float)gr.dims;
  float* __restrict__ out = static_cast<float*>(L.out);
  const int nbatch = (zend - zbeg + ZC - 1) / ZC;
  const int nitems = (nbatch + 1) * DPT;  // item q: batch q / DPT - 1 (-1: prologue), dir q % DPT

  if (lane == 0) {
    for (int r = 0; r < R; ++r) mbar_init(smem_u32(&mbar[g * R + r]), 1);
  }
  if (g == 0 && lane == 0) *abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  float* my_ring = ring + (size_t)g * R * SLOT;
  bool alive = true;
  int issued = 0;
  // issue item q into slot q % R (lane 0)
  auto issue = [&](int q) {
    if (q >= nitems || !alive) return;
    issued = q + 1;
    __syncwarp();
    if (lane == 0) {
      const int slot = q % R;
      const uint32_t bar = smem_u32(&mbar[g * R + slot]);
      const int i = g * DPT + (q % DPT);
      if (i < L.N) {
        fence_proxy_async();
        const int oct = __float_as_int(t.au[i].w);
        const int s = (oct & 4) ? 1 : 0;
        const int b = q / DPT - 1;
        // first plane of the box (padded coordinates: plane z + 1)
        const int zp = (b < 0 ? zbeg - 1 : zbeg + b * ZC) + s + 1;
        const int yp = (oct & 2) ? y + 1 : y;  // lower of the two rows (padded)
        mbar_arrive_tx(bar, BOXX * 2 * ZC * 4);
        tma_load_3d(smem_u32(my_ring + (size_t)slot * SLOT), &tmap, x0,
                    yp, i * gr.PZ + zp, bar);
      } else {
        mbar_arrive_tx(bar, 0);
      }
    }
  };
  auto wait_item = [&](int q) -> bool {
    if (!alive || *reinterpret_cast<volatile int*>(abort_flag)) {
      alive = false;
      return false;
    }
    if (!mbar_wait(smem_u32(&mbar[g * R + q % R]), (uint32_t)((q / R) & 1), L.err)) {
      *reinterpret_cast<volatile int*>(abort_flag) = 1;
      alive = false;
      return false;
    }
    return true;
  };

  int q = 0;
  for (int r = 0; r < R - 1; ++r) issue(r);

  // window column of the lane's pair: x - (x0 - 2)
  const int wc = 2 + 2 * lane;
  float2 carry[DPT];
#pragma unroll
  for (int k = 0; k < DPT; ++k) {
    issue(q + R - 1);
    carry[k] = make_float2(0.f, 0.f);
    const int i = g * DPT + k;
    if (wait_item(q) && i < L.N) {
      const float4 au = t.au[i];
      const int oct = __float_as_int(au.w);
      const bool xneg = oct & 1;
      const float* slot = my_ring + (size_t)(q % R) * SLOT;
      const float* r0 = slot + ((oct & 2) ? 0 : BOXX);   // own row
      const float* r1 = slot + ((oct & 2) ? BOXX : 0);   // upwind row
      const int uc = xneg ? wc + 2 : wc - 1;
      const float2 v0 = *reinterpret_cast<const float2*>(r0 + wc);
      const float2 v1 = *reinterpret_cast<const float2*>(r1 + wc);
      const float u0 = r0[uc], u1 = r1[uc];
      const float2 w0 = xneg ? make_float2(v0.y, u0) : make_float2(u0, v0.x);
      const float2 w1 = xneg ? make_float2(v1.y, u1) : make_float2(u1, v1.x);
      const float2 ax = f2s(au.x), ay = f2s(au.y);
      carry[k] = f2lerp(ay, f2lerp(ax, w1, v1), f2lerp(ax, w0, v0));
    }
    ++q;
  }

  double bud_a = 0.0, bud_b = 0.0;
  for (int b = 0; b < nbatch; ++b) {
    const int zb = zbeg + b * ZC;
    const int nb = min(ZC, zend - zb);
    float2 aE[ZC], aX[ZC], aY[ZC], aZ[ZC];
#pragma unroll
    for (int j = 0; j < ZC; ++j) aE[j] = aX[j] = aY[j] = aZ[j] = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      issue(q + R - 1);
      const int i = g * DPT + k;
      if (wait_item(q) && i < L.N) {
        const float4 au = t.au[i];
        const float4 nw = t.nw[i];
        const int oct = __float_as_int(au.w);
        const bool xneg = oct & 1;
        const int uc = xneg ? wc + 2 : wc - 1;
        const float2 ax = f2s(au.x), ay = f2s(au.y);
        const float2 az = f2s((oct & 4) ? 1.f - au.z : au.z);
        const float2 nx2 = f2s(nw.x), ny2 = f2s(nw.y), nz2 = f2s(nw.z);
        const float* slot = my_ring + (size_t)(q % R) * SLOT;
        const int o0 = (oct & 2) ? 0 : BOXX, o1 = (oct & 2) ? BOXX : 0;
#pragma unroll
        for (int j = 0; j < ZC; ++j) {
          const float* r0 = slot + j * 2 * BOXX + o0;
          const float* r1 = slot + j * 2 * BOXX + o1;
          const float2 v0 = *reinterpret_cast<const float2*>(r0 + wc);
          const float2 v1 = *reinterpret_cast<const float2*>(r1 + wc);
          const float u0 = r0[uc], u1 = r1[uc];
          const float2 w0 = xneg ? make_float2(v0.y, u0) : make_float2(u0, v0.x);
          const float2 w1 = xneg ? make_float2(v1.y, u1) : make_float2(u1, v1.x);
          const float2 Bn = f2lerp(ay, f2lerp(ax, w1, v1), f2lerp(ax, w0, v0));
          // I* = (1 - a_z) B(z) + a_z B(z - sgn n^z); the carried plane is B(z - 1)
          // for sgn = +1 and B(z) for sgn = -1
          const float2 r = f2lerp(az, carry[k], Bn);
          carry[k] = Bn;
          Ist[((size_t)i * ZC + j) * 32 + lane] = r;
          aE[j] = f2add(aE[j], r);
          aX[j] = f2fma(nx2, r, aX[j]);
          aY[j] = f2fma(ny2, r, aY[j]);
          aZ[j] = f2fma(nz2, r, aZ[j]);
        }
      }
      ++q;
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
    for (int item = g * 32 + lane; item < nb * 32; item += G * 32) {
      const int j = item >> 5, l = item & 31;
      float2 E = make_float2(0.f, 0.f), Fx = E, Fy = E, Fz = E;
      for (int qq = 0; qq < G; ++qq) {
        const float2* p = part + (((size_t)qq * ZC + j) * 4) * 32 + l;
        E = f2add(E, p[0]);
        Fx = f2add(Fx, p[32]);
        Fy = f2add(Fy, p[64]);
        Fz = f2add(Fz, p[96]);
      }
      const int xs = x0 + 2 * l;
      const long long site = ((long long)(zb + j) * gr.ny + y) * nx + xs;
      float2 o[5];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const bool ok = xs + h < nx;
        const long long st = ok ? site + h : 0;
        const float ka = fld(cf.ka, cf.ka_s, st), k0 = fld(cf.k0, cf.k0_s, st);
        const float lam = fld(cf.lam, cf.lam_s, st), eta = fld(cf.eta, cf.eta_s, st);
        const float Es = h ? E.y : E.x;
        const Coef c = collide_scalars(L.collision, L.lambda_iters, L.dt, inv_d, ka, k0, lam,
                                       eta, Es, h ? Fx.y : Fx.x, h ? Fy.y : Fy.x, h ? Fz.y : Fz.x);
        const float v[5] = {c.alpha, c.c0, c.c1x, c.c1y, c.c1z};
#pragma unroll
        for (int u = 0; u < 5; ++u) (h ? o[u].y : o[u].x) = v[u];
        if (ok) {
          bud_a += (double)Es;
          bud_b += (double)c.Enew;
        }
      }
      float2* cp = coef + ((size_t)j * 5) * 32 + l;
#pragma unroll
      for (int u = 0; u < 5; ++u) cp[u * 32] = o[u];
    }
    __syncthreads();
    float2 al[ZC], c0[ZC], c1x[ZC], c1y[ZC], c1z[ZC];
#pragma unroll
    for (int j = 0; j < ZC; ++j) {
      const float2* cp = coef + ((size_t)j * 5) * 32 + lane;
      al[j] = cp[0];
      c0[j] = cp[32];
      c1x[j] = cp[64];
      c1y[j] = cp[96];
      c1z[j] = cp[128];
    }
    if (alive) {
      // interior sites with no ghost mirror take the float2 fast path
      const bool yz_edge = (gr.periodic[1] && (y == 0 || y == gr.ny - 1)) || gr.periodic[2];
      const bool x_edge = gr.periodic[0] && (xa == 0 || xa + 1 >= nx - 1);
#pragma unroll
      for (int k = 0; k < DPT; ++k) {
        const int i = g * DPT + k;
        if (i < L.N) {
          const float4 nw = t.nw[i];
          const float2 nx2 = f2s(nw.x), ny2 = f2s(nw.y), nz2 = f2s(nw.z), w2 = f2s(nw.w);
#pragma unroll
          for (int j = 0; j < ZC; ++j) {
            if (j < nb && in0) {
              const int z = zb + j;
              const float2 r = Ist[((size_t)i * ZC + j) * 32 + lane];
              const float2 eq =
                  f2fma(nz2, c1z[j], f2fma(ny2, c1y[j], f2fma(nx2, c1x[j], c0[j])));
              const float2 o = f2fma(al[j], r, f2mul(w2, eq));
              const bool mirror = x_edge || (yz_edge && (y == 0 || y == gr.ny - 1 ||
                                                         z == 0 || z == nz - 1));
              if (in1 && !mirror) {
                *reinterpret_cast<float2*>(out + pidx(gr, i, z, y, xa)) = o;
              } else {
                store_pop(out, gr, i, z, y, xa, o.x);
                if (in1) store_pop(out, gr, i, z, y, xa + 1, o.y);
              }
            }
          }
        }
      }
    }
  }
  // every issued copy must land before the CTA's shared memory is released
  for (int qq = q; qq < issued; ++qq)
    mbar_wait(smem_u32(&mbar[g * R + qq % R]), (uint32_t)((qq / R) & 1), L.err);
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
size_t tma_smem(int G) {
  return sizeof(float) * (size_t)G * R * slot_floats<ZC>() +
         sizeof(float2) * 32 * ((size_t)G * DPT * ZC + (size_t)G * ZC * 4 + ZC * 5) + 8 * G * R +
         16;
}

template <int DPT, int ZC, int R>
cudaError_t launch_tma(const StepLaunch& L, const StaticCoef& c, const DirTable& t, int G,
                       int zchunk, cudaStream_t s, int* nblocks) {
  dim3 block(32, G);
  dim3 grid((L.g.nx + 63) / 64, L.g.ny, (L.g.nz + zchunk - 1) / zchunk);
  const long long nb_ = (long long)grid.x * grid.y * grid.z;
  if (L.budget_partials && nb_ > L.partials_cap) return cudaErrorInvalidValue;
  if (nblocks) *nblocks = (int)nb_;
  const size_t smem = tma_smem<DPT, ZC, R>(G);
  if (smem > 227 * 1024 || !L.tmap_in) return cudaErrorInvalidValue;
  // the opt-in shared-memory size is a per-device function attribute
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && !(attr_set >> dev & 1ull)) {
    const cudaError_t e = cudaFuncSetAttribute(
        k_tma_static<DPT, ZC, R>, cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024);
    if (e != cudaSuccess) return e;
    attr_set |= 1ull << dev;
  }
  k_tma_static<DPT, ZC, R><<<grid, block, smem, s>>>(*L.tmap_in, L, c, t, zchunk);
  return cudaGetLastError();
}

}  // namespace

int tma_planes_per_batch(int N) { return N <= 48 ? 2 : 1; }

// Direction groups of 8 (N <= 48, 2 planes per batch) or 21 (larger sets,
// 1 plane per batch: shared memory holds I* of every direction of a batch);
// z chunks of 32 planes.
cudaError_t launch_tma_static(const StepLaunch& L, const StaticCoef& c, const DirTable& t,
                              cudaStream_t s, int* nblocks) {
  const int N = L.N;
  const int zchunk = 32;
  if (N <= 48) return launch_tma<8, 2, 4>(L, c, t, (N + 7) / 8, zchunk, s, nblocks);
  return launch_tma<21, 1, 4>(L, c, t, (N + 20) / 21, zchunk, s, nblocks);
}

bool make_pop_tensor_map(CUtensorMap* map, const Grid& g, int N, void* base, int zc,
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
  const cuuint64_t dims[3] = {(cuuint64_t)g.PX, (cuuint64_t)g.PY, (cuuint64_t)g.PZ * N};
  const cuuint64_t strides[2] = {(cuuint64_t)g.PX * 4, (cuuint64_t)g.plane * 4};
  const cuuint32_t box[3] = {(cuuint32_t)BOXX, 2, (cuuint32_t)zc};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box,
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
