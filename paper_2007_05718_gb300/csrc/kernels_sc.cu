// Pipelined fused stream + collide step for a static fluid (single problem),
// float32 or 16-bit population storage, fed by TMA tensor tiles.  Weih et
// al. 2020: Sec. 3.3, Eqs. (interp), (rte_implicit), (collision-step).
//
// Tiles, boxes and the z-sweep with the carried plane are those of the
// first-generation kernels (kernels_tma.cu, kernels_tma16.cu): a CTA owns 64
// x-sites of one row over a chunk of planes, each lane an x-pair, and the
// stream warp g the DPT directions g DPT .. of one upwind (row, plane) class,
// one box of DPT directions x 2 rows x ZC planes per batch.  What changes is
// who waits for whom.
//
// The moment reduction of a batch (sum over all directions of a site) needs
// every stream warp, and the collision of the batch needs the reduction.  In
// the first-generation kernels every warp waited twice per batch at CTA
// barriers while a few warps summed the partial moments and formed the
// collision scalars.  Here the reduction runs on dedicated coefficient warps
// (one per plane of a batch) and the stream warps store batch b - 1 while
// the coefficient warps work on batch b:
//
//   stream warp, batch b:  issue TMA(b + 1); wait TMA(b); stream(b) -> I*(b)
//                          in registers; [C(b - 1)]; write partials(b);
//                          arrive P(b); store batch b - 1 with coef(b - 1)
//   coef warp, batch b:    [P(b)]; sum partials(b); collision scalars ->
//                          coef(b) (double-buffered); budget / E, F epilogue
//                          / 16-bit E field; arrive C(b)
//
// P and C are named hardware barriers; [X] marks a wait.  Every warp of the
// CTA walks the same sequence of batches (the round-robin tile order), so
// every barrier phase collects the whole CTA.  A stream warp holds the
// streamed values of two batches in registers (I*(b - 1) until its store
// after the stream pass of b).  The partial moments have one buffer: the
// stream warps write partials(b) only after C(b - 1), i.e. after the
// coefficient warps have read partials(b - 1).  Bounded waits: the TMA
// waits give up after about 2 s, set the device error word and let the
// batch run on with stale (in-bounds) data, so that every warp still takes
// part in every barrier phase.
#include <algorithm>

#include "lb_rt_internal.h"
#include "tma_common.cuh"

#include <cudaTypedefs.h>

namespace lbrt {

namespace {

using namespace tma;

constexpr int kBarP = 1;  // partial moments of a batch written (stream -> coef)
constexpr int kBarC = 2;  // collision scalars of a batch ready (coef -> stream)
constexpr float kEpsE = 1e-30f;
constexpr int kBoxH = 72;  // 16-bit box columns (the first-generation 16-bit box)

__device__ __forceinline__ void bar_sync_n(int id, int n) {
  asm volatile("bar.sync %0, %1;" ::"r"(id), "r"(n) : "memory");
}
__device__ __forceinline__ void bar_arrive_n(int id, int n) {
  asm volatile("bar.arrive %0, %1;" ::"r"(id), "r"(n) : "memory");
}

template <class ST> struct SV;
template <> struct SV<float> {
  static constexpr int BOX = BOXX;  // float32 box columns
  static constexpr bool F32 = true;
};
template <> struct SV<__half> {
  static constexpr int BOX = kBoxH;
  static constexpr bool F32 = false;
  using T2 = __half2;
  static __device__ __forceinline__ float2 to2(T2 v) { return __half22float2(v); }
  static __device__ __forceinline__ float to1(__half v) { return __half2float(v); }
  static __device__ __forceinline__ T2 from2(float2 v) { return __float22half2_rn(v); }
};
template <> struct SV<__nv_bfloat16> {
  static constexpr int BOX = kBoxH;
  static constexpr bool F32 = false;
  using T2 = __nv_bfloat162;
  static __device__ __forceinline__ float2 to2(T2 v) { return __bfloat1622float2(v); }
  static __device__ __forceinline__ float to1(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ T2 from2(float2 v) { return __float22bfloat162_rn(v); }
};

// Per-direction constants as pre-broadcast pairs for the packed float32 x 2
// arithmetic: s0 = (a_x, a_x, a_y, a_y), s1 = (a_z', a_z', n_x, n_x),
// s2 = (n_y, n_y, n_z, n_z), o0 = (w, w, w n_x, w n_x), o1 = (w n_y, w n_y,
// w n_z, w n_z); sh = offset of the x-upwind pair (-1 for sgn n^x = +1, +1
// otherwise); inert = padding entry.  The products and the order of every
// sum are those of the first-generation kernels, so a problem gives the same
// bits here and in a batched launch.
struct DirSC {
  float4 s0, s1, s2, o0, o1;
  int sh, inert, pad0, pad1;
};

template <class ST, int DPT, int ZC>
__host__ __device__ constexpr int sc_slot_bytes() {
  return ((SV<ST>::BOX * DPT * 2 * ZC * (int)sizeof(ST) + 127) / 128) * 128;
}
template <int ZC>
__host__ __device__ constexpr int sc_eslot_floats() {
  return ((kBoxH * 3 * (ZC + 1) * 4 + 127) / 128) * 32;
}
constexpr int kEring = 3;  // E boxes in flight (16-bit storage)

// Shared-memory layout (bytes): ring [G][2][SLOT] | E ring [3][ESLOT] |
// partials [G][ZC][4][64] f32 | coef [2][ZC][5][64] f32 | dirs [G DPT] |
// mbar [G][2] | ebar [3] | budget [ZC][2] double | abort flag
template <class ST, int DPT, int ZC>
__host__ __device__ constexpr size_t sc_smem_bytes(int G) {
  return (size_t)G * 2 * sc_slot_bytes<ST, DPT, ZC>() +
         (SV<ST>::F32 ? 0 : (size_t)kEring * sc_eslot_floats<ZC>() * 4) +
         (size_t)G * ZC * 4 * 64 * 4 + 2 * ZC * 5 * 64 * 4 + sizeof(DirSC) * (size_t)G * DPT +
         8 * (size_t)G * 2 + 8 * kEring + 16 * ZC + 16;
}

// Store context of a batch, kept until its deferred store: the output
// address of the lane's pair in direction i0 of plane zb + 1 (padded), the
// plane of j = 0, and flag bits (bit 0: fast path; bit 1: a lane of the warp
// writes an x ghost column; bit 2: the row is on a periodic y face; bits
// 8 + j: plane j lies in the tile; bits 16 + j: plane j is on a periodic z
// face); the tile index for the general path.
template <class ST>
struct BatchCtx {
  ST* base;
  int zb, flags, ti;
};

template <class ST, int MODE, bool PER, int DPT, int ZC, int MAXT, int REGS>
__global__ void __launch_bounds__(MAXT) __maxnreg__(REGS)
k_sc(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap emap,
     const __grid_constant__ ProblemDesc P, int ntiles, unsigned* err, const DirTable t) {
  constexpr bool F32 = SV<ST>::F32;
  constexpr bool MOM = MODE == 2;
  constexpr int BOX = SV<ST>::BOX;
  constexpr int SLOT = sc_slot_bytes<ST, DPT, ZC>();
  constexpr int ESLOT = sc_eslot_floats<ZC>();
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int NW = blockDim.y;       // warps: G stream + ZC coefficient
  const int G = NW - ZC;
  const int NT = NW * 32;
  const int lane = threadIdx.x, g = threadIdx.y;
  unsigned char* ring = smem_raw;
  float* ering = reinterpret_cast<float*>(ring + (size_t)G * 2 * SLOT);
  float* part = ering + (F32 ? 0 : kEring * ESLOT);
  float* coef = part + (size_t)G * ZC * 4 * 64;
  DirSC* dirs = reinterpret_cast<DirSC*>(coef + 2 * ZC * 5 * 64);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(dirs + G * DPT);
  unsigned long long* ebar = mbar + G * 2;
  double* bsum = reinterpret_cast<double*>(ebar + kEring);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bsum + 2 * ZC);

  const Grid& gr = P.g;
  const int nx = gr.nx, ny = gr.ny, nz = gr.nz;
  const int nxb = (nx + 63) / 64;

  for (int i = g * 32 + lane; i < G * DPT; i += NT) {
    const float4 au = t.au[i], nw = t.nw[i];
    const int oct = __float_as_int(au.w);
    const float azw = (oct & 4) ? 1.f - au.z : au.z;
    DirSC d;
    d.s0 = make_float4(au.x, au.x, au.y, au.y);
    d.s1 = make_float4(azw, azw, nw.x, nw.x);
    d.s2 = make_float4(nw.y, nw.y, nw.z, nw.z);
    const float wx = nw.w * nw.x, wy = nw.w * nw.y, wz = nw.w * nw.z;
    d.o0 = make_float4(nw.w, nw.w, wx, wx);
    d.o1 = make_float4(wy, wy, wz, wz);
    d.sh = (oct & 1) ? 1 : -1;
    d.inert = oct & 8;
    d.pad0 = d.pad1 = 0;
    dirs[i] = d;
  }
  if (g < G && lane == 0)
    for (int r = 0; r < 2; ++r) mbar_init(smem_u32(&mbar[g * 2 + r]), 1);
  if (!F32 && g == 0 && lane == 0)
    for (int r = 0; r < kEring; ++r) mbar_init(smem_u32(&ebar[r]), 1);
  if (g == 0 && lane == 0) *abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  __syncthreads();

  // the batch cursor every warp walks: tile ti (round-robin), item m of M
  int ti = blockIdx.x, m = 0;
  TileGeom tg = tile_geom(ti, nxb, ny, nz, P.nzc);
  int M = tile_items<ZC>(tg.zlen);
  auto advance = [&]() {
    if (++m == M) {
      m = 0;
      ti += gridDim.x;
      if (ti < ntiles) {
        tg = tile_geom(ti, nxb, ny, nz, P.nzc);
        M = tile_items<ZC>(tg.zlen);
      }
    }
  };
  const float inv_d = 1.f / (float)gr.dims;

  if (g >= G) {
    // ------------------------------------------------------------------
    // coefficient warp u = g - G: plane j = u of every batch, lane = x-pair
    // ------------------------------------------------------------------
    const int j = g - G;
    const StaticCoef& cf = P.cf;
    float bud_a = 0.f, bud_b = 0.f;
    double bud_da = 0.0, bud_db = 0.0;
    int q = 0;
    for (; ti < ntiles; advance(), ++q) {
      const int zb = tg.zbeg - 1 + m * ZC;
      const int z = zb + j, y = tg.y;
      const int xa = tg.x0 + 2 * lane;
      const bool zin = z >= tg.zbeg && z < tg.zbeg + tg.zlen;
      const bool v0 = zin && xa < nx, v1 = zin && xa + 1 < nx;
      const long long st0 = v0 ? ((long long)z * ny + y) * nx + xa : 0;
      const long long st1 = v1 ? st0 + 1 : 0;
      // fields first: their latency overlaps the wait for the partials
      const float ka0 = fld(cf.ka, cf.ka_s, st0), ka1 = fld(cf.ka, cf.ka_s, st1);
      const float k00 = fld(cf.k0, cf.k0_s, st0), k01 = fld(cf.k0, cf.k0_s, st1);
      const float lm0 = fld(cf.lam, cf.lam_s, st0), lm1 = fld(cf.lam, cf.lam_s, st1);
      const float et0 = fld(cf.eta, cf.eta_s, st0), et1 = fld(cf.eta, cf.eta_s, st1);
      bar_sync_n(kBarP, NT);
      float2 E = make_float2(0.f, 0.f), X = E, Y = E, Z = E;
      const float2* pp = reinterpret_cast<const float2*>(part + (size_t)j * 4 * 64) + lane;
#pragma unroll 4
      for (int w = 0; w < G; ++w) {
        const float2* p = pp + (size_t)w * ZC * 4 * 32;
        E = f2add(E, p[0]);
        X = f2add(X, p[32]);
        Y = f2add(Y, p[64]);
        Z = f2add(Z, p[96]);
      }
      const Coef c0 = collide_scalars(P.collision, P.lambda_iters, P.dt, inv_d, ka0, k00, lm0, et0,
                                      E.x, X.x, Y.x, Z.x);
      const Coef c1 = collide_scalars(P.collision, P.lambda_iters, P.dt, inv_d, ka1, k01, lm1, et1,
                                      E.y, X.y, Y.y, Z.y);
      float2* cp = reinterpret_cast<float2*>(coef + ((size_t)(q & 1) * ZC + j) * 5 * 64) + lane;
      if constexpr (F32) {
        cp[0] = make_float2(c0.alpha, c1.alpha);
        cp[32] = make_float2(c0.c0, c1.c0);
        cp[64] = make_float2(c0.c1x, c1.c1x);
        cp[96] = make_float2(c0.c1y, c1.c1y);
        cp[128] = make_float2(c0.c1z, c1.c1z);
      } else {
        // q' = f' / E^' - 1: the float32 coefficients scaled by 1 / E^'
        const float e0 = fmaxf(c0.Enew, kEpsE), e1 = fmaxf(c1.Enew, kEpsE);
        const float r0 = __fdividef(1.f, e0), r1 = __fdividef(1.f, e1);
        cp[0] = make_float2(c0.alpha * r0, c1.alpha * r1);
        cp[32] = make_float2(fmaf(c0.c0, r0, -1.f), fmaf(c1.c0, r1, -1.f));
        cp[64] = make_float2(c0.c1x * r0, c1.c1x * r1);
        cp[96] = make_float2(c0.c1y * r0, c1.c1y * r1);
        cp[128] = make_float2(c0.c1z * r0, c1.c1z * r1);
        float* eout = P.e_out;
        // E^' of the site and of its periodic ghost mirrors
        const bool face = has_mirror(gr, z, y, xa) || (v1 && has_mirror(gr, z, y, xa + 1));
        if (!face) {
          float* ep = eout + ((long long)(z + 1) * gr.PY + (y + 1)) * gr.PX + xa + GL;
          if (v1) *reinterpret_cast<float2*>(ep) = make_float2(e0, e1);
          else if (v0) ep[0] = e0;
        } else {
          auto put_e = [&](int x, float val) {
            int xs[3], ys[3], zs_[3];
            const int nxs = mirrors(x, gr.nx, gr.periodic[0], GL, xs);
            const int nys = mirrors(y, gr.ny, gr.periodic[1], 1, ys);
            const int nzs = mirrors(z, gr.nz, gr.periodic[2], 1, zs_);
            for (int a = 0; a < nzs; ++a)
              for (int b = 0; b < nys; ++b)
                for (int c = 0; c < nxs; ++c)
                  eout[((long long)zs_[a] * gr.PY + ys[b]) * gr.PX + xs[c]] = val;
          };
          if (v0) put_e(xa, e0);
          if (v1) put_e(xa + 1, e1);
        }
      }
      if (v0) {
        bud_a += E.x;
        bud_b += c0.Enew;
      }
      if (v1) {
        bud_a += E.y;
        bud_b += c1.Enew;
      }
      if constexpr (MOM) {
        // moments of I' = alpha I* + w (c0 + n . c1) for an isotropic table
        // (sum w = 1, sum w n = 0, sum w n n = Id / d): E' = alpha E* + c0,
        // F' = alpha F* + c1 / d
        if (P.mom_E) {
          if (v0) P.mom_E[st0] = c0.Enew;
          if (v1) P.mom_E[st1] = c1.Enew;
        }
        if (P.mom_F) {
          const long long S = gr.sites;
          if (v0) {
            P.mom_F[st0] = fmaf(c0.alpha, X.x, c0.c1x * inv_d);
            P.mom_F[S + st0] = fmaf(c0.alpha, Y.x, c0.c1y * inv_d);
            P.mom_F[2 * S + st0] = fmaf(c0.alpha, Z.x, c0.c1z * inv_d);
          }
          if (v1) {
            P.mom_F[st1] = fmaf(c1.alpha, X.y, c1.c1x * inv_d);
            P.mom_F[S + st1] = fmaf(c1.alpha, Y.y, c1.c1y * inv_d);
            P.mom_F[2 * S + st1] = fmaf(c1.alpha, Z.y, c1.c1z * inv_d);
          }
        }
      }
      if (P.budget_partials) {
        bud_da += (double)bud_a;
        bud_db += (double)bud_b;
      }
      bud_a = bud_b = 0.f;
      bar_arrive_n(kBarC, NT);
    }
    if (P.budget_partials) {
      for (int s = 16; s > 0; s >>= 1) {
        bud_da += __shfl_xor_sync(0xffffffffu, bud_da, s);
        bud_db += __shfl_xor_sync(0xffffffffu, bud_db, s);
      }
      if (lane == 0) {
        atomicAdd(P.budget_partials + 2 * blockIdx.x, bud_da);
        atomicAdd(P.budget_partials + 2 * blockIdx.x + 1, bud_db);
      }
    }
    return;
  }

  // --------------------------------------------------------------------
  // stream warp g: directions i0 .. i0 + DPT - 1 (one upwind class)
  // --------------------------------------------------------------------
  const int i0 = g * DPT;
  const int oct0 = __float_as_int(t.au[i0].w);
  const bool yneg = oct0 & 2;
  const int zs = (oct0 & 4) ? 1 : 0;
  const int row_own = yneg ? 0 : 1, row_up = yneg ? 1 : 0;  // rows of a population box
  const int erow_up = yneg ? 2 : 0;                          // rows of the E box: y-1, y, y+1
  unsigned inert_mask = 0;
#pragma unroll
  for (int k = 0; k < DPT; ++k) inert_mask |= dirs[i0 + k].inert ? 1u << k : 0u;
  unsigned char* my_ring = ring + (size_t)g * 2 * SLOT;
  bool alive = true;
  int waited = 0;  // items whose copies have landed

  // issue the copies of batch q (tile t, item mm of a tile with geometry gq)
  int q_is = 0;  // batches issued
  auto issue_item = [&](int t, int mm, const TileGeom& gq) {
    if (t >= ntiles || !alive) return;
    const int slot = q_is & 1;
    __syncwarp();
    if (lane == 0) {
      const uint32_t bar = smem_u32(&mbar[g * 2 + slot]);
      fence_proxy_async();
      mbar_arrive_tx(bar, BOX * DPT * 2 * ZC * (int)sizeof(ST));
      tma_load_4d(smem_u32(my_ring + (size_t)slot * SLOT), &tmap, gq.x0, i0, yneg ? gq.y + 1 : gq.y,
                  gq.zbeg + zs + mm * ZC, bar);
      if (!F32 && g == 0) {
        const int es = q_is % kEring;
        const uint32_t eb = smem_u32(&ebar[es]);
        mbar_arrive_tx(eb, kBoxH * 3 * (ZC + 1) * 4);
        tma_load_3d(smem_u32(ering + (size_t)es * ESLOT), &emap, gq.x0, gq.y, gq.zbeg + mm * ZC, eb);
      }
    }
    ++q_is;
  };
  // the batch after the current one (same tile, or the CTA's next tile)
  auto issue_next = [&]() {
    if (m + 1 < M) {
      issue_item(ti, m + 1, tg);
    } else {
      const int tn = ti + gridDim.x;
      if (tn < ntiles) issue_item(tn, 0, tile_geom(tn, nxb, ny, nz, P.nzc));
    }
  };
  // the outcome is made warp-uniform, so that every later warp-collective
  // step (syncwarp, votes) sees the whole warp on the same path
  auto wait_item = [&](int q) {
    if (!__all_sync(0xffffffffu, alive && !*abort_flag)) {
      alive = false;
      return;
    }
    const uint32_t par = (uint32_t)((q >> 1) & 1);
    bool ok = mbar_wait(smem_u32(&mbar[g * 2 + (q & 1)]), par, err);
    if (!F32 && ok) ok = mbar_wait(smem_u32(&ebar[q % kEring]), (uint32_t)((q / kEring) & 1), err);
    if (!__all_sync(0xffffffffu, ok)) {
      if (lane == 0) *abort_flag = 1;
      alive = false;
      return;
    }
    waited = q + 1;
  };

  ST* __restrict__ out = static_cast<ST*>(P.out);
  const int wc = 2 + 2 * lane;  // box column of the lane's pair

  // deferred store of one batch
  auto store_batch = [&](const float2 (&Is)[DPT][ZC], const BatchCtx<ST>& bc, int par) {
    float2 al[ZC], c0[ZC], c1x[ZC], c1y[ZC], c1z[ZC];
#pragma unroll
    for (int j = 0; j < ZC; ++j) {
      const float2* c = reinterpret_cast<const float2*>(coef + ((size_t)par * ZC + j) * 5 * 64) + lane;
      al[j] = c[0];
      c0[j] = c[32];
      c1x[j] = c[64];
      c1y[j] = c[96];
      c1z[j] = c[128];
    }
    if (!alive) return;
    // I' = alpha I* + w c0 + (w n) . c1 (float32); with 16-bit storage the
    // coefficients are scaled by 1 / E^' and f = I / w, so q' = A' f* +
    // c0' + n . c1'
    auto value = [&](int k, int j) {
      const DirSC& d = dirs[i0 + k];
      if constexpr (F32) {
        const float4 o0 = d.o0, o1 = d.o1;
        const float2 w2 = make_float2(o0.x, o0.y), wx2 = make_float2(o0.z, o0.w);
        const float2 wy2 = make_float2(o1.x, o1.y), wz2 = make_float2(o1.z, o1.w);
        const float2 eq =
            f2fma(wz2, c1z[j], f2fma(wy2, c1y[j], f2fma(wx2, c1x[j], f2mul(w2, c0[j]))));
        return f2fma(al[j], Is[k][j], eq);
      } else {
        const float4 s1 = d.s1, s2 = d.s2;
        const float2 nx2 = make_float2(s1.z, s1.w), ny2 = make_float2(s2.x, s2.y),
                     nz2 = make_float2(s2.z, s2.w);
        return f2fma(al[j], Is[k][j], f2fma(nz2, c1z[j], f2fma(ny2, c1y[j], f2fma(nx2, c1x[j], c0[j]))));
      }
    };
    auto put2 = [&](ST* p, float2 o) {
      if constexpr (F32) *reinterpret_cast<float2*>(p) = o;
      else *reinterpret_cast<typename SV<ST>::T2*>(p) = SV<ST>::from2(o);
    };
    if (bc.flags & 1) {
      // every lane a full interior pair, every plane of the batch in the
      // tile, no periodic y or z face: one pair store per direction and plane
      // (plus the x ghost column on a periodic x edge)
      ST* p = bc.base;
      const long long si = gr.si, sz = gr.sz;
      // x ghost column of a periodic x edge: the lane holding x = nx - 1
      // mirrors it into column GL - 1 (from o.y when x = nx - 1 is the
      // second site of its pair), the lane holding x = 0 into column nx + GL
      const bool xg = PER && (bc.flags & 2);
      int gx_off = 0;
      bool gx_lane = false, gx_y = false;
      if (PER && xg) {
        const int xa = (bc.ti % nxb) * 64 + 2 * lane;
        const bool gx_lo = xa == nx - 1 || xa + 1 == nx - 1;
        gx_lane = gx_lo || xa == 0;
        gx_off = gx_lo ? GL - 1 - (xa + GL) : nx + GL - (xa + GL);
        gx_y = gx_lo && xa + 1 == nx - 1;
      }
#pragma unroll
      for (int k = 0; k < DPT; ++k) {
        if (!(inert_mask >> k & 1u)) {
#pragma unroll
          for (int j = 0; j < ZC; ++j) {
            const float2 o = value(k, j);
            ST* d = p + j * sz;
            put2(d, o);
            if (PER && xg) {
              if (gx_lane) {
                if constexpr (F32) d[gx_off] = gx_y ? o.y : o.x;
                else {
                  const typename SV<ST>::T2 h = SV<ST>::from2(o);
                  d[gx_off] = gx_y ? h.y : h.x;
                }
              }
            }
          }
        }
        p += si;
      }
      return;
    }
    // general path: ragged rows, periodic faces (every row / plane image)
    const TileGeom gq = tile_geom(bc.ti, nxb, ny, nz, P.nzc);
    const int y = gq.y, xa = gq.x0 + 2 * lane;
    if (xa >= nx) return;
    const bool in1 = xa + 1 < nx;
    const bool gx_lo = gr.periodic[0] && (xa == nx - 1 || xa + 1 == nx - 1);
    const bool gx_hi = gr.periodic[0] && xa == 0;
    const bool lo_from_y = xa + 1 == nx - 1;
#pragma unroll
    for (int k = 0; k < DPT; ++k) {
      if (inert_mask >> k & 1u) continue;
#pragma unroll
      for (int j = 0; j < ZC; ++j) {
        if (!(bc.flags >> (8 + j) & 1)) continue;
        const int z = bc.zb + j;
        const float2 o = value(k, j);
        ST hx, hy;
        if constexpr (F32) {
          hx = o.x;
          hy = o.y;
        } else {
          const typename SV<ST>::T2 h = SV<ST>::from2(o);
          hx = h.x;
          hy = h.y;
        }
        const ST hlo = lo_from_y ? hy : hx;
        const int rows[3] = {y + 1, (gr.periodic[1] && y == ny - 1) ? 0 : -1,
                             (gr.periodic[1] && y == 0) ? ny + 1 : -1};
        const int planes[3] = {z + 1, (gr.periodic[2] && z == nz - 1) ? 0 : -1,
                               (gr.periodic[2] && z == 0) ? nz + 1 : -1};
#pragma unroll 1
        for (int cmb = 0; cmb < 9; ++cmb) {
          const int rr = rows[cmb % 3], pp = planes[cmb / 3];
          if (rr < 0 || pp < 0) continue;
          ST* b = out + (long long)(i0 + k) * gr.si + (long long)pp * gr.sz + (long long)rr * gr.sy;
          b[xa + GL] = hx;
          if (in1) b[xa + GL + 1] = hy;
          if (gx_lo) b[GL - 1] = hlo;
          if (gx_hi) b[nx + GL] = hx;
        }
      }
    }
  };

  auto make_ctx = [&]() {
    BatchCtx<ST> bc;
    const int zb = tg.zbeg - 1 + m * ZC;
    const int xa = tg.x0 + 2 * lane;
    const int y = tg.y;
    int flags = 0;
    bool plain = true;
#pragma unroll
    for (int j = 0; j < ZC; ++j) {
      const int z = zb + j;
      const bool zok = z >= tg.zbeg && z < tg.zbeg + tg.zlen;
      const bool zf = gr.periodic[2] && (z == 0 || z == nz - 1);
      flags |= (zok ? 1 : 0) << (8 + j);
      flags |= (zf ? 1 : 0) << (16 + j);
      plain = plain && zok && !zf;
    }
    const bool yf = gr.periodic[1] && (y == 0 || y == ny - 1);
    plain = plain && !yf;
    const bool full = __all_sync(0xffffffffu, xa + 1 < nx);
    const bool xg = __any_sync(0xffffffffu, gr.periodic[0] && (xa == 0 || xa == nx - 1 || xa + 1 == nx - 1));
    // the fast path writes the x ghost column only in the periodic
    // specialisation; the plain one sends x-edge batches to the general path
    if (full && plain && (PER || !xg)) flags |= 1;
    if (xg) flags |= 2;
    if (yf) flags |= 4;
    bc.flags = flags;
    bc.zb = zb;
    bc.ti = ti;
    bc.base = out + (long long)i0 * gr.si + (long long)(zb + 1) * gr.sz + (long long)(y + 1) * gr.sy +
              xa + GL;
    return bc;
  };

  float2 carry[DPT];
#pragma unroll
  for (int k = 0; k < DPT; ++k) carry[k] = make_float2(0.f, 0.f);
  float2 IsA[DPT][ZC], IsB[DPT][ZC];
  BatchCtx<ST> ctx{};  // store context of the previous batch

  // one batch: stream into `cur`, then store `prev` (the previous batch)
  auto batch = [&](int q, float2 (&cur)[DPT][ZC], const float2 (&prev)[DPT][ZC]) {
    issue_next();
    wait_item(q);
    float2 aE[ZC], aX[ZC], aY[ZC], aZ[ZC];
#pragma unroll
    for (int j = 0; j < ZC; ++j) aE[j] = aX[j] = aY[j] = aZ[j] = make_float2(0.f, 0.f);
    const unsigned char* slot = my_ring + (size_t)(q & 1) * SLOT;
    if constexpr (F32) {
      const float* own = reinterpret_cast<const float*>(slot) + row_own * DPT * BOX + wc;
      const float* up = reinterpret_cast<const float*>(slot) + row_up * DPT * BOX + wc;
#pragma unroll
      for (int k = 0; k < DPT; ++k) {
        const DirSC& d = dirs[i0 + k];
        const float4 s0 = d.s0, s1 = d.s1, s2 = d.s2;
        const float2 ax = make_float2(s0.x, s0.y), ay = make_float2(s0.z, s0.w);
        const float2 az = make_float2(s1.x, s1.y), nx2 = make_float2(s1.z, s1.w);
        const float2 ny2 = make_float2(s2.x, s2.y), nz2 = make_float2(s2.z, s2.w);
        const float* ownS = own + d.sh;
        const float* upS = up + d.sh;
#pragma unroll
        for (int j = 0; j < ZC; ++j) {
          const int off = (j * 2 * DPT + k) * BOX;
          // Eq. (interp) as nested lerps: x on both rows, then y, then z
          // against the carried plane
          const float2 P0 = *reinterpret_cast<const float2*>(own + off);
          const float2 S0 = make_float2(ownS[off], ownS[off + 1]);
          const float2 P1 = *reinterpret_cast<const float2*>(up + off);
          const float2 S1 = make_float2(upS[off], upS[off + 1]);
          const float2 X0 = f2fma(ax, f2sub(S0, P0), P0);
          const float2 X1 = f2fma(ax, f2sub(S1, P1), P1);
          const float2 Bn = f2fma(ay, f2sub(X1, X0), X0);
          const float2 r = f2fma(az, f2sub(carry[k], Bn), Bn);
          carry[k] = Bn;
          cur[k][j] = r;
          aE[j] = f2add(aE[j], r);
          aX[j] = f2fma(nx2, r, aX[j]);
          aY[j] = f2fma(ny2, r, aY[j]);
          aZ[j] = f2fma(nz2, r, aZ[j]);
        }
      }
    } else {
      using T2 = typename SV<ST>::T2;
      const ST* sl = reinterpret_cast<const ST*>(slot);
      const float* es = ering + (size_t)(q % kEring) * ESLOT;
      // E^ of the lane's pair and of its two x-neighbours, own and upwind row
      float2 EPo[ZC], EPu[ZC];
      float Emo[ZC], Epo[ZC], Emu[ZC], Epu[ZC];
#pragma unroll
      for (int j = 0; j < ZC; ++j) {
        const float* eo = es + ((j + zs) * 3 + 1) * kBoxH + wc;
        const float* eu = es + ((j + zs) * 3 + erow_up) * kBoxH + wc;
        EPo[j] = *reinterpret_cast<const float2*>(eo);
        EPu[j] = *reinterpret_cast<const float2*>(eu);
        Emo[j] = eo[-1];
        Epo[j] = eo[2];
        Emu[j] = eu[-1];
        Epu[j] = eu[2];
      }
#pragma unroll
      for (int k = 0; k < DPT; ++k) {
        const DirSC& d = dirs[i0 + k];
        const float4 s0 = d.s0, s1 = d.s1, s2 = d.s2;
        const float2 ax = make_float2(s0.x, s0.y), ay = make_float2(s0.z, s0.w);
        const float2 az = make_float2(s1.x, s1.y);
        const float4 o0 = d.o0, o1 = d.o1;
        const float2 w2 = make_float2(o0.x, o0.y), wx2 = make_float2(o0.z, o0.w);
        const float2 wy2 = make_float2(o1.x, o1.y), wz2 = make_float2(o1.z, o1.w);
        // Eq. (interp) on the decoded f = E^ (1 + q); the x-upwind side
        // decides which edge value completes the shifted pair
        auto pass = [&](auto xneg) {
#pragma unroll
          for (int j = 0; j < ZC; ++j) {
            const ST* po = sl + ((j * 2 + row_own) * DPT + k) * kBoxH + wc;
            const ST* pu = sl + ((j * 2 + row_up) * DPT + k) * kBoxH + wc;
            const float2 qo = SV<ST>::to2(*reinterpret_cast<const T2*>(po));
            const float2 qu = SV<ST>::to2(*reinterpret_cast<const T2*>(pu));
            const float2 fo = f2fma(EPo[j], qo, EPo[j]);
            const float2 fu = f2fma(EPu[j], qu, EPu[j]);
            float2 So, Su;
            if (decltype(xneg)::value) {
              const float eo = fmaf(Epo[j], SV<ST>::to1(po[2]), Epo[j]);
              const float eu = fmaf(Epu[j], SV<ST>::to1(pu[2]), Epu[j]);
              So = make_float2(fo.y, eo);
              Su = make_float2(fu.y, eu);
            } else {
              const float eo = fmaf(Emo[j], SV<ST>::to1(po[-1]), Emo[j]);
              const float eu = fmaf(Emu[j], SV<ST>::to1(pu[-1]), Emu[j]);
              So = make_float2(eo, fo.x);
              Su = make_float2(eu, fu.x);
            }
            const float2 X0 = f2fma(ax, f2sub(So, fo), fo);
            const float2 X1 = f2fma(ax, f2sub(Su, fu), fu);
            const float2 Bn = f2fma(ay, f2sub(X1, X0), X0);
            const float2 r = f2fma(az, f2sub(carry[k], Bn), Bn);
            carry[k] = Bn;
            cur[k][j] = r;
            aE[j] = f2fma(w2, r, aE[j]);
            aX[j] = f2fma(wx2, r, aX[j]);
            aY[j] = f2fma(wy2, r, aY[j]);
            aZ[j] = f2fma(wz2, r, aZ[j]);
          }
        };
        if (d.sh > 0) pass(std::true_type());
        else pass(std::false_type());
      }
    }
    if (q > 0) bar_sync_n(kBarC, NT);  // coef(q - 1) ready; partials(q - 1) read
    {
      float2* pw = reinterpret_cast<float2*>(part + (size_t)g * ZC * 4 * 64) + lane;
#pragma unroll
      for (int j = 0; j < ZC; ++j) {
        pw[j * 128] = aE[j];
        pw[j * 128 + 32] = aX[j];
        pw[j * 128 + 64] = aY[j];
        pw[j * 128 + 96] = aZ[j];
      }
    }
    bar_arrive_n(kBarP, NT);
    if (q > 0) store_batch(prev, ctx, (q - 1) & 1);
    ctx = make_ctx();
    advance();
  };

  if (ti < ntiles) issue_item(ti, 0, tg);  // batch 0; every batch issues the one after it
  int q = 0;
  while (ti < ntiles) {
    batch(q, IsA, IsB);
    ++q;
    if (ti >= ntiles) break;
    batch(q, IsB, IsA);
    ++q;
  }
  if (q > 0) {
    bar_sync_n(kBarC, NT);
    if (q & 1) store_batch(IsA, ctx, (q - 1) & 1);
    else store_batch(IsB, ctx, (q - 1) & 1);
  }
  // copies still in flight (only after a failed wait) land before exit
  for (int qq = waited; qq < q_is; ++qq) {
    mbar_wait(smem_u32(&mbar[g * 2 + (qq & 1)]), (uint32_t)((qq >> 1) & 1), err);
    if (!F32 && g == 0) mbar_wait(smem_u32(&ebar[qq % kEring]), (uint32_t)((qq / kEring) & 1), err);
  }
}

template <class ST, int MODE, bool PER, int DPT, int ZC, int MAXT, int REGS>
cudaError_t sc_attr() {
  static unsigned long long done = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && (done >> dev & 1ull)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(k_sc<ST, MODE, PER, DPT, ZC, MAXT, REGS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024 - 1024);
  if (e == cudaSuccess && dev < 64) done |= 1ull << dev;
  return e;
}

template <class ST, int DPT, int ZC, int MAXT, int REGS>
cudaError_t sc_occupancy(int G, int* per_sm) {
  const size_t smem = sc_smem_bytes<ST, DPT, ZC>(G);
  const int threads = 32 * (G + ZC);
  // the moments-epilogue variant (MODE 2) exists for float32 storage only
  constexpr int M2 = SV<ST>::F32 ? 2 : 0;
  int r[4] = {0, 0, 0, 0};
  cudaError_t e = sc_attr<ST, 0, false, DPT, ZC, MAXT, REGS>();
  if (e == cudaSuccess) e = sc_attr<ST, 0, true, DPT, ZC, MAXT, REGS>();
  if (e == cudaSuccess) e = sc_attr<ST, M2, false, DPT, ZC, MAXT, REGS>();
  if (e == cudaSuccess) e = sc_attr<ST, M2, true, DPT, ZC, MAXT, REGS>();
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r[0], k_sc<ST, 0, false, DPT, ZC, MAXT, REGS>,
                                                      threads, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r[1], k_sc<ST, 0, true, DPT, ZC, MAXT, REGS>,
                                                      threads, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r[2], k_sc<ST, M2, false, DPT, ZC, MAXT, REGS>,
                                                      threads, smem);
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&r[3], k_sc<ST, M2, true, DPT, ZC, MAXT, REGS>,
                                                      threads, smem);
  *per_sm = std::min(std::min(r[0], r[1]), std::min(r[2], r[3]));
  return e;
}

template <class ST, int DPT, int ZC, int MAXT, int REGS>
cudaError_t sc_launch(const StepLaunch& L, const StaticCoef& c, const DirTable& t, cudaStream_t s,
                      int* nblocks) {
  const int G = L.N / DPT;
  if (!L.tmap_in || G < 1 || G * DPT != L.N || 32 * (G + ZC) > MAXT || L.nzc < 1 ||
      L.nzc > L.g.nz || L.ctas < 1)
    return cudaErrorInvalidValue;
  if (!SV<ST>::F32 && (!L.tmap_e || !L.e_out)) return cudaErrorInvalidValue;
  if (L.budget_partials && L.ctas > L.partials_cap) return cudaErrorInvalidValue;
  const size_t smem = sc_smem_bytes<ST, DPT, ZC>(G);
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  const bool per = L.g.periodic[0] || L.g.periodic[1] || L.g.periodic[2];
  const bool mom = SV<ST>::F32 && (L.mom_E || L.mom_F);
  ProblemDesc P{};
  P.g = L.g;
  P.out = L.out;
  P.e_out = L.e_out;
  P.cf = c;
  P.dt = L.dt;
  P.collision = L.collision;
  P.lambda_iters = L.lambda_iters;
  P.nzc = L.nzc;
  P.tile_start = 0;
  P.ntiles = (L.g.nx + 63) / 64 * L.g.ny * L.nzc;
  P.budget_partials = L.budget_partials;
  P.mom_E = mom ? L.mom_E : nullptr;
  P.mom_F = mom ? L.mom_F : nullptr;
  if (nblocks) *nblocks = L.ctas;
  const CUtensorMap emap = SV<ST>::F32 ? CUtensorMap{} : *L.tmap_e;
  const dim3 block(32, G + ZC);
  cudaError_t e;
#define LBRT_SC_GO(MODE_, PER_)                                                                 \
  do {                                                                                          \
    e = sc_attr<ST, MODE_, PER_, DPT, ZC, MAXT, REGS>();                                        \
    if (e != cudaSuccess) return e;                                                             \
    k_sc<ST, MODE_, PER_, DPT, ZC, MAXT, REGS><<<L.ctas, block, smem, s>>>(*L.tmap_in, emap, P, \
                                                                           P.ntiles, L.err, t); \
  } while (0)
  constexpr int M2 = SV<ST>::F32 ? 2 : 0;  // moments epilogue: float32 only
  if (mom && per) LBRT_SC_GO(M2, true);
  else if (mom) LBRT_SC_GO(M2, false);
  else if (per) LBRT_SC_GO(0, true);
  else LBRT_SC_GO(0, false);
#undef LBRT_SC_GO
  return cudaGetLastError();
}

// Tile plans of the pipelined kernel (directions per warp, planes per batch,
// thread cap including the coefficient warps, registers per thread), in
// order of preference.  A stream warp keeps the carried plane and two
// batches of streamed values in registers: 96 per thread give two 10-warp
// CTAs per SM (ico42: 45 internal directions, 9 stream warps + 1
// coefficient warp).  The 162-direction set (16 stream warps + 1 coefficient
// warp) would leave 96 registers per thread (resident warps are counted in
// groups of 4, so 17 warps take 20 warps' worth), which do not hold two
// batches; it runs the first-generation kernel.
#define LBRT_SC_PLANS(X) \
  X(5, 1, 320, 96)       \
  X(4, 1, 544, 96)

template <class ST>
cudaError_t sc_launch_typed(const StepLaunch& L, const StaticCoef& c, const DirTable& t, cudaStream_t s,
                            int* nblocks) {
#define LBRT_SC_L(D, Z, T, B) \
  if (L.dpt == D && L.zc == Z) return sc_launch<ST, D, Z, T, B>(L, c, t, s, nblocks);
  LBRT_SC_PLANS(LBRT_SC_L)
#undef LBRT_SC_L
  return cudaErrorInvalidValue;
}

template <class ST>
cudaError_t sc_occupancy_typed(int dpt, int zc, int G, int* per_sm) {
#define LBRT_SC_O(D, Z, T, B) \
  if (dpt == D && zc == Z) return sc_occupancy<ST, D, Z, T, B>(G, per_sm);
  LBRT_SC_PLANS(LBRT_SC_O)
#undef LBRT_SC_O
  return cudaErrorInvalidValue;
}

}  // namespace

#define LBRT_SC_ROW(D, Z, T, B) {D, Z, T},
const int kTilePlansSC[][3] = {LBRT_SC_PLANS(LBRT_SC_ROW)};
#undef LBRT_SC_ROW
const int kNumTilePlansSC = sizeof(kTilePlansSC) / sizeof(kTilePlansSC[0]);

size_t step_tile_smem_sc(int storage, int dpt, int zc, int stream_warps) {
#define LBRT_SC_S(D, Z, T, B)                                                  \
  if (dpt == D && zc == Z)                                                     \
    return storage == ST_F32 ? sc_smem_bytes<float, D, Z>(stream_warps)        \
                             : sc_smem_bytes<__half, D, Z>(stream_warps);
  LBRT_SC_PLANS(LBRT_SC_S)
#undef LBRT_SC_S
  return (size_t)-1;
}

cudaError_t occupancy_sc(int storage, int dpt, int zc, int stream_warps, int* per_sm) {
  if (storage == ST_F32) return sc_occupancy_typed<float>(dpt, zc, stream_warps, per_sm);
  if (storage == ST_F16) return sc_occupancy_typed<__half>(dpt, zc, stream_warps, per_sm);
  if (storage == ST_BF16) return sc_occupancy_typed<__nv_bfloat16>(dpt, zc, stream_warps, per_sm);
  return cudaErrorInvalidValue;
}

cudaError_t launch_sc_static(const StepLaunch& L, const StaticCoef& c, const DirTable& t, int storage,
                             cudaStream_t s, int* nblocks) {
  if (storage == ST_F32) return sc_launch_typed<float>(L, c, t, s, nblocks);
  if (storage == ST_F16) return sc_launch_typed<__half>(L, c, t, s, nblocks);
  if (storage == ST_BF16) return sc_launch_typed<__nv_bfloat16>(L, c, t, s, nblocks);
  return cudaErrorInvalidValue;
}

}  // namespace lbrt
