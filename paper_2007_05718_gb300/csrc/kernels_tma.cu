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
#include <numeric>

#include "lb_rt_internal.h"
#include "tma_common.cuh"

#include <cudaTypedefs.h>

namespace lbrt {

namespace {

using namespace tma;

// Per-direction constants in shared memory, as pre-broadcast pairs for the
// packed float32 x 2 arithmetic: s0 = (a_x, a_x, a_y, a_y), s1 = (a_z', a_z',
// n_x, n_x), s2 = (n_y, n_y, n_z, n_z) for the stream pass (a_z' the weight of
// the carried plane), o0 = (w, w, w n_x, w n_x), o1 = (w n_y, w n_y, w n_z,
// w n_z) for the output; sh = offset (floats) of the x-upwind pair of the
// lane's own pair (-1 for sgn n^x = +1, +1 otherwise); inert = padding entry.
struct DirConst {
  float4 s0, s1, s2, o0, o1;
  int sh, inert, pad0, pad1;
};

// MODE 0: one problem, `one` and `tmap1` in the parameter space.
// MODE 1 (batched): `table[nprob]` in device memory; each CTA copies the
// descriptor of its current tile into shared memory.
// MODE 2: as MODE 0, and the coefficient units also store E and F of the
// new state (one.mom_E, one.mom_F); a separate instantiation keeps the
// plain step's code unchanged.
// PER: some problem of the launch has a periodic axis (ghost columns,
// mirror rows and planes are written by the fast store path); all-vacuum
// launches use the plain store loop.
// The body runs on CTA `cta` of `ncta` persistent CTAs with G warps; PART:
// the block belongs to a launch shared by two tile plans (k_step_f32_pair).
// XP: complete the x-upwind pair with one 4-byte shared load behind a branch
// on the x sign (faster for vacuum faces and for periodic faces when the
// grid rotates the CTAs over the x-blocks; see plan_static_grid).
// ROT: permute the x-blocks of each round of tiles (tile_rot); compiled in
// for the single-problem plans of one CTA per SM, whose grid is a multiple of
// the x-blocks (the plans of two or more CTAs per SM get a coprime grid).
template <int MODE, bool PER, int DPT, int ZC, int R, bool PART, bool XP, bool ROT>
__device__ __forceinline__ void step_f32_body(const CUtensorMap& tmap1, const ProblemDesc& one,
                                              const ProblemDesc* __restrict__ table, int nprob,
                                              int ntiles, unsigned* err, const DirTable& t,
                                              const int cta, const int ncta, const int G) {
  constexpr bool BATCH = MODE == 1;
  constexpr bool MOM = MODE == 2;
  constexpr int SLOT = slot_floats<DPT, ZC>();
  static_assert(SLOT >= ZC * 4 * 64, "the partial moments must fit in a consumed slot");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x, g = threadIdx.y;
  __shared__ ProblemDesc pd[BATCH ? 2 : 1];
  // shared layout: ring [G][R][SLOT] | coef [ZC][5][64] | dirs [N] DirConst |
  // mbar [G][R] | budget [2 ZC][2] double | abort flag
  float* ring = reinterpret_cast<float*>(smem_raw);
  float* coef = ring + (size_t)G * R * SLOT;
  DirConst* dirs = reinterpret_cast<DirConst*>(coef + ZC * 5 * 64);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(dirs + G * DPT);
  double* bsum = reinterpret_cast<double*>(mbar + G * R);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bsum + 4 * ZC);

  const int i0 = g * DPT;
  // the warp's row / plane class (uniform over its directions)
  const int oct0 = __float_as_int(t.au[i0].w);
  const bool yneg = oct0 & 2;
  const int zs = (oct0 & 4) ? 1 : 0;
  const int row_own = yneg ? 0 : 1, row_up = yneg ? 1 : 0;
  const int nunits = 2 * ZC;  // coefficient units: (plane, half row) pairs of a batch

  for (int i = g * 32 + lane; i < G * DPT; i += G * 32) {
    const float4 au = t.au[i], nw = t.nw[i];
    const int oct = __float_as_int(au.w);
    const float azw = (oct & 4) ? 1.f - au.z : au.z;
    DirConst d;
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
  if (lane == 0) {
    for (int r = 0; r < R; ++r) mbar_init(smem_u32(&mbar[g * R + r]), 1);
  }
  if (g == 0 && lane == 0) *abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  cta_sync<PART>(32 * G);
  unsigned inert_mask = 0;  // padding directions of this warp
#pragma unroll
  for (int k = 0; k < DPT; ++k) inert_mask |= dirs[i0 + k].inert ? 1u << k : 0u;

  float* my_ring = ring + (size_t)g * R * SLOT;
  bool alive = true;
  int issued = 0, waited = 0;
  // issue cursor (tile, item), ahead of the consumer by up to R - 1 items
  int is_t = cta, is_p = 0, is_m = 0, is_M = 0, is_x0 = 0, is_yp = 0, is_zp = 0;
  const CUtensorMap* is_map = &tmap1;
  auto issue_seek = [&]() {
    if (is_t < ntiles) {
      if constexpr (BATCH) {
        while (is_p < nprob && is_t >= table[is_p].tile_start + table[is_p].ntiles) ++is_p;
        if (is_p >= nprob) {  // inconsistent table: stop issuing (the consumer reports it)
          is_t = ntiles;
          return;
        }
        is_map = table[is_p].tmap;
      }
      const ProblemDesc& D = BATCH ? table[is_p] : one;
      const int nxb_i = (D.g.nx + 63) / 64, rel_i = is_t - D.tile_start;
      const TileGeom tg = tile_geom(rel_i, nxb_i, D.g.ny, D.g.nz, D.nzc,
                                    ROT ? tile_rot(rel_i, nxb_i, ncta, D.g.periodic[0]) : 0);
      is_M = tile_items<ZC>(tg.zlen);
      is_x0 = tg.x0;
      is_yp = yneg ? tg.y + 1 : tg.y;  // lower padded row of the box
      is_zp = tg.zbeg + zs;            // padded plane of B(zbeg - 1), shifted for sgn n^z < 0
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
      tma_load_4d(smem_u32(my_ring + (size_t)slot * SLOT), is_map, is_x0, i0, is_yp,
                  is_zp + is_m * ZC, bar);
    }
    ++issued;
    if (++is_m == is_M) {
      is_m = 0;
      is_t += ncta;
      issue_seek();
    }
    return true;
  };
  auto wait_item = [&](int q) -> bool {
    if (!alive || *abort_flag) {
      alive = false;
      return false;
    }
    if (!mbar_wait(smem_u32(&mbar[g * R + q % R]), (uint32_t)((q / R) & 1), err)) {
      *abort_flag = 1;
      alive = false;
      return false;
    }
    waited = q + 1;
    return true;
  };
  const int wc = 2 + 2 * lane;  // window column of the lane's pair in a box row

  while (issued < R - 1 && issue()) {
  }

  float2 carry[DPT];
#pragma unroll
  for (int k = 0; k < DPT; ++k) carry[k] = make_float2(0.f, 0.f);
  float bud_a = 0.f, bud_b = 0.f;  // FP32 per batch, folded into FP64 below
  double bud_da = 0.0, bud_db = 0.0;
  int q = 0;   // items consumed
  int tk = 0;  // tiles taken by this CTA
  int cp = 0;  // problem of the current tile
  for (int ti = cta; ti < ntiles; ti += ncta, ++tk) {
    const ProblemDesc* Pp = &one;
    if constexpr (BATCH) {
      while (cp < nprob && ti >= table[cp].tile_start + table[cp].ntiles) ++cp;
      if (cp >= nprob) {  // the tile counts do not add up: report, stop (uniform per CTA)
        if (g == 0 && lane == 0) atomicOr(err, 4u);
        break;
      }
      ProblemDesc* dst = &pd[tk & 1];
      if (g == 0) {
        const int* src = reinterpret_cast<const int*>(&table[cp]);
        for (int w = lane; w < (int)(sizeof(ProblemDesc) / 4); w += 32)
          reinterpret_cast<int*>(dst)[w] = src[w];
      }
      cta_sync<PART>(32 * G);
      Pp = dst;
    }
    const ProblemDesc& P = *Pp;
    const Grid& gr = P.g;
    const int nx = gr.nx, ny = gr.ny, nz = gr.nz;
    const float inv_d = 1.f / (float)gr.dims;
    float* __restrict__ out = static_cast<float*>(P.out);
    const StaticCoef& cf = P.cf;
    const int nxb_t = (nx + 63) / 64, rel_t = ti - P.tile_start;
    const TileGeom tg = tile_geom(rel_t, nxb_t, ny, nz, P.nzc,
                                  ROT ? tile_rot(rel_t, nxb_t, ncta, gr.periodic[0]) : 0);
    const int x0 = tg.x0, y = tg.y, zbeg = tg.zbeg, zend = tg.zbeg + tg.zlen;
    const int M = tile_items<ZC>(tg.zlen);
    const int xa = x0 + 2 * lane;  // the lane's pair (xa, xa + 1)
    const bool in0 = xa < nx, in1 = xa + 1 < nx;
    // x ghost columns this lane mirrors into (periodic x): column GL - 1
    // holds x = nx - 1, column nx + GL holds x = 0
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
      const int zb = zbeg - 1 + m * ZC;  // output plane of j = 0
      // coefficient fields of this warp's first unit, loaded before the
      // stream pass so that their latency overlaps it
      float pka = 0.f, pk0 = 0.f, plam = 0.f, peta = 0.f;
      if (g < nunits) {
        const int j = g >> 1, x = x0 + ((g & 1) << 5) + lane, z = zb + j;
        const bool v = x < nx && z >= zbeg && z < zend;
        const long long st = v ? ((long long)z * ny + y) * nx + x : 0;
        pka = fld(cf.ka, cf.ka_s, st);
        pk0 = fld(cf.k0, cf.k0_s, st);
        plam = fld(cf.lam, cf.lam_s, st);
        peta = fld(cf.eta, cf.eta_s, st);
      }
      while (issued < q + R && issue()) {
      }
      // after a failed wait the slot holds stale (finite, in-bounds) data:
      // the pass runs anyway and the error word reports the step as failed
      wait_item(q);
      float* slot = my_ring + (size_t)(q % R) * SLOT;
      const float* own = slot + row_own * DPT * BOXX + wc;
      const float* up = slot + row_up * DPT * BOXX + wc;
      float2 Is[DPT][ZC];
      float2 aE[ZC], aX[ZC], aY[ZC], aZ[ZC];
#pragma unroll
      for (int j = 0; j < ZC; ++j) aE[j] = aX[j] = aY[j] = aZ[j] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < DPT; ++k) {
        const DirConst& d = dirs[i0 + k];
        const float4 s0 = d.s0, s1 = d.s1, s2 = d.s2;
        const float2 ax = make_float2(s0.x, s0.y), ay = make_float2(s0.z, s0.w);
        const float2 az = make_float2(s1.x, s1.y), nx2 = make_float2(s1.z, s1.w);
        const float2 ny2 = make_float2(s2.x, s2.y), nz2 = make_float2(s2.z, s2.w);
        const bool xneg = d.sh > 0;  // uniform over the warp
        const float* ownS = own + d.sh;
        const float* upS = up + d.sh;
#pragma unroll
        for (int j = 0; j < ZC; ++j) {
          const int off = (j * 2 * DPT + k) * BOXX;
          // Eq. (interp) as nested lerps: x on both rows, then y, then z
          // against the carried plane (B(z - 1) for sgn n^z = +1, B(z + 1)
          // otherwise, the box being shifted by one plane for the latter).
          // The x-upwind pair shares one value with the lane's own pair: with
          // XP one more 4-byte load completes it (3 % faster for vacuum
          // faces, 3-5 % with periodic faces when the CTAs rotate over the
          // x-blocks); otherwise both values are loaded (without the rotation
          // the branch made the periodic kernel 5 % slower)
          const float2 P0 = *reinterpret_cast<const float2*>(own + off);
          const float2 P1 = *reinterpret_cast<const float2*>(up + off);
          float2 S0, S1;
          if constexpr (!XP) {
            S0 = make_float2(ownS[off], ownS[off + 1]);
            S1 = make_float2(upS[off], upS[off + 1]);
          } else if (xneg) {
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
          Is[k][j] = r;
          aE[j] = f2add(aE[j], r);
          aX[j] = f2fma(nx2, r, aX[j]);
          aY[j] = f2fma(ny2, r, aY[j]);
          aZ[j] = f2fma(nz2, r, aZ[j]);
        }
      }
      // the slot has been read: it now holds this warp's partial moments
      // [ZC][E, Fx, Fy, Fz][64 sites]
      __syncwarp();
#pragma unroll
      for (int j = 0; j < ZC; ++j) {
        float2* p = reinterpret_cast<float2*>(slot + j * 4 * 64) + lane;
        p[0] = aE[j];
        p[32] = aX[j];
        p[64] = aY[j];
        p[96] = aZ[j];
      }
      cta_sync<PART>(32 * G);
      // coefficient units: unit u = (plane u / 2, sites 32 (u % 2) .. + 31)
      for (int u = g; u < nunits; u += G) {
        const int j = u >> 1, f = ((u & 1) << 5) + lane;
        const int x = x0 + f, z = zb + j;
        const bool v = x < nx && z >= zbeg && z < zend;
        float ka = pka, k0 = pk0, lam = plam, eta = peta;
        if (u != g) {
          const long long st = v ? ((long long)z * ny + y) * nx + x : 0;
          ka = fld(cf.ka, cf.ka_s, st);
          k0 = fld(cf.k0, cf.k0_s, st);
          lam = fld(cf.lam, cf.lam_s, st);
          eta = fld(cf.eta, cf.eta_s, st);
        }
        const int s = q % R;
        float E = 0.f, Fx = 0.f, Fy = 0.f, Fz = 0.f;
        for (int qq = 0; qq < G; ++qq) {
          const float* p = ring + ((size_t)qq * R + s) * SLOT + j * 4 * 64 + f;
          E += p[0];
          Fx += p[64];
          Fy += p[128];
          Fz += p[192];
        }
        const Coef cc =
            collide_scalars(P.collision, P.lambda_iters, P.dt, inv_d, ka, k0, lam, eta, E, Fx, Fy, Fz);
        float* c = coef + j * 5 * 64 + f;
        c[0] = cc.alpha;
        c[64] = cc.c0;
        c[128] = cc.c1x;
        c[192] = cc.c1y;
        c[256] = cc.c1z;
        if (v) {
          bud_a += E;
          bud_b += cc.Enew;
          if constexpr (MOM) {
            // moments of I' = alpha I* + w (c0 + n . c1) for an isotropic
            // table (sum w = 1, sum w n = 0, sum w n n = Id / d):
            // E' = alpha E* + c0 = Enew, F' = alpha F* + c1 / d
            const long long st = ((long long)z * ny + y) * nx + x;
            if (one.mom_E) one.mom_E[st] = cc.Enew;
            if (one.mom_F) {
              one.mom_F[st] = fmaf(cc.alpha, Fx, cc.c1x * inv_d);
              one.mom_F[gr.sites + st] = fmaf(cc.alpha, Fy, cc.c1y * inv_d);
              one.mom_F[2 * gr.sites + st] = fmaf(cc.alpha, Fz, cc.c1z * inv_d);
            }
          }
        }
      }
      cta_sync<PART>(32 * G);
      if (!BATCH && one.budget_partials && g < nunits) {
        bud_da += (double)bud_a;
        bud_db += (double)bud_b;
        bud_a = bud_b = 0.f;
      }
      // I_i^{n+1} = alpha I*_i + w_i c0 + (w_i n_i) . c1, direction-major so
      // that each direction's constants are read once per batch
      float2 al[ZC], c0[ZC], c1x[ZC], c1y[ZC], c1z[ZC];
#pragma unroll
      for (int j = 0; j < ZC; ++j) {
        const float2* c = reinterpret_cast<const float2*>(coef + j * 5 * 64) + lane;
        al[j] = c[0];
        c0[j] = c[32];
        c1x[j] = c[64];
        c1y[j] = c[96];
        c1z[j] = c[128];
      }
      bool zok[ZC], zface[ZC];
      // the fast path writes one mirror row / plane at a periodic face; an
      // extent of 1 on a periodic axis (two mirrors) takes the general path
      bool batch_plain = !(y_face && ny == 1);
#pragma unroll
      for (int j = 0; j < ZC; ++j) {
        const int z = zb + j;
        zok[j] = z >= zbeg && z < zend;
        zface[j] = gr.periodic[2] && (z == 0 || z == nz - 1);
        batch_plain = batch_plain && zok[j] && !(zface[j] && nz == 1);
      }
      // offsets (elements) of the mirror row / plane of a face row / plane
      const int yface_rows = (y == ny - 1 ? 0 : ny + 1) - (y + 1);
      // fast path: every plane of the batch in the tile, no periodic y/z
      // face, every lane a full interior pair; a warp with a lane on a
      // periodic x edge takes the variant that also writes the x ghost column
      const bool fast = __all_sync(0xffffffffu, in0 && in1) && batch_plain;
      const bool xghost = __any_sync(0xffffffffu, gx_lo || gx_hi);
      bool done_fast = false;
      if constexpr (!PER) {
        if (alive && fast) {
          // interior batch: one float2 store per direction and plane
          float* base = orow + (long long)(zb + 1) * gr.sz;
#pragma unroll
          for (int k = 0; k < DPT; ++k) {
            if (inert_mask >> k & 1u) continue;  // padding direction: its populations stay 0
            const DirConst& d = dirs[i0 + k];
            const float4 o0 = d.o0, o1 = d.o1;
            const float2 w2 = make_float2(o0.x, o0.y), wx2 = make_float2(o0.z, o0.w);
            const float2 wy2 = make_float2(o1.x, o1.y), wz2 = make_float2(o1.z, o1.w);
#pragma unroll
            for (int j = 0; j < ZC; ++j) {
              const float2 eq =
                  f2fma(wz2, c1z[j], f2fma(wy2, c1y[j], f2fma(wx2, c1x[j], f2mul(w2, c0[j]))));
              *reinterpret_cast<float2*>(base + (long long)k * gr.si + (long long)j * gr.sz) =
                  f2fma(al[j], Is[k][j], eq);
            }
          }
          done_fast = true;
        }
      } else {
        if (alive && fast) {
          // periodic edges: the same stores plus the x ghost column and one
          // mirror row / plane image
          float* base = orow + (long long)(zb + 1) * gr.sz;
#pragma unroll
          for (int k = 0; k < DPT; ++k) {
            if (inert_mask >> k & 1u) continue;
            const DirConst& d = dirs[i0 + k];
            const float4 o0 = d.o0, o1 = d.o1;
            const float2 w2 = make_float2(o0.x, o0.y), wx2 = make_float2(o0.z, o0.w);
            const float2 wy2 = make_float2(o1.x, o1.y), wz2 = make_float2(o1.z, o1.w);
#pragma unroll
            for (int j = 0; j < ZC; ++j) {
              const float2 eq =
                  f2fma(wz2, c1z[j], f2fma(wy2, c1y[j], f2fma(wx2, c1x[j], f2mul(w2, c0[j]))));
              const float2 o = f2fma(al[j], Is[k][j], eq);
              float* dst = base + (long long)k * gr.si + (long long)j * gr.sz;
              auto put = [&](float* dd) {
                *reinterpret_cast<float2*>(dd) = o;
                if (xghost && gx_any) dd[gx_off] = gx_y ? o.y : o.x;  // one predicated store
              };
              put(dst);
              if (y_face) put(dst + (long long)yface_rows * gr.sy);  // warp-uniform
              if (zface[j]) {
                const int z = zb + j;
                const long long zd = (long long)((z == nz - 1 ? 0 : nz + 1) - (z + 1)) * gr.sz;
                put(dst + zd);
                if (y_face) put(dst + zd + (long long)yface_rows * gr.sy);
              }
            }
          }
          done_fast = true;
        }
      }
      if (!done_fast && alive && in0) {
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
          if (inert_mask >> k & 1u) continue;
          const DirConst& d = dirs[i0 + k];
          const float4 o0 = d.o0, o1 = d.o1;
          const float2 w2 = make_float2(o0.x, o0.y), wx2 = make_float2(o0.z, o0.w);
          const float2 wy2 = make_float2(o1.x, o1.y), wz2 = make_float2(o1.z, o1.w);
#pragma unroll
          for (int j = 0; j < ZC; ++j) {
            if (!zok[j]) continue;
            const int z = zb + j;
            const float2 eq = f2fma(wz2, c1z[j], f2fma(wy2, c1y[j], f2fma(wx2, c1x[j], f2mul(w2, c0[j]))));
            const float2 o = f2fma(al[j], Is[k][j], eq);
            const float vlo = lo_from_y ? o.y : o.x;
            if (!(y_face || zface[j])) {
              float* base = orow + (long long)k * gr.si + (long long)(z + 1) * gr.sz;
              if (in1) *reinterpret_cast<float2*>(base) = o;
              else base[0] = o.x;
              if (gx_lo) base[GL - 1 - (xa + GL)] = vlo;
              if (gx_hi) base[nx + GL - (xa + GL)] = o.x;
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
  // copies still in flight (only after a failed wait) must land before the
  // CTA's shared memory is released; each slot has at most one outstanding
  for (int qq = waited; qq < issued; ++qq) {
    mbar_wait(smem_u32(&mbar[g * R + qq % R]), (uint32_t)((qq / R) & 1), err);
  }
  if (!BATCH && one.budget_partials) {
    for (int s = 16; s > 0; s >>= 1) {
      bud_da += __shfl_xor_sync(0xffffffffu, bud_da, s);
      bud_db += __shfl_xor_sync(0xffffffffu, bud_db, s);
    }
    if (lane == 0 && g < nunits) {
      bsum[2 * g] = bud_da;
      bsum[2 * g + 1] = bud_db;
    }
    cta_sync<PART>(32 * G);
    if (g == 0 && lane == 0) {
      double a = 0.0, b = 0.0;
      for (int w = 0; w < min(G, nunits); ++w) {
        a += bsum[2 * w];
        b += bsum[2 * w + 1];
      }
      atomicAdd(one.budget_partials + 2 * cta, a);
      atomicAdd(one.budget_partials + 2 * cta + 1, b);
    }
  }
}

template <int MODE, bool PER, int DPT, int ZC, int R, int MAXT, int REGS>
__global__ void __launch_bounds__(MAXT) __maxnreg__(REGS)
k_step_f32(const __grid_constant__ CUtensorMap tmap1, const __grid_constant__ ProblemDesc one,
           const ProblemDesc* __restrict__ table, int nprob, int ntiles, unsigned* err,
           const DirTable t) {
  // the one-load x pair: vacuum faces, or a single-problem launch, whose
  // CTAs rotate over the x-blocks with a periodic x axis (a grid coprime to
  // the x-blocks, or tile_rot); a batched launch does not rotate
  constexpr bool XP = !PER || MODE != 1;
  constexpr bool ROT = PER && MODE != 1 && 2 * MAXT * REGS > 65536;
  step_f32_body<MODE, PER, DPT, ZC, R, false, XP, ROT>(tmap1, one, table, nprob, ntiles, err, t,
                                                       blockIdx.x, gridDim.x, blockDim.y);
}

// One batched launch over the problems of two groups with different tile
// plans (the 42- and 162-direction icosahedral sets): CTAs 0 .. ctas_a - 1
// walk group A's tiles with GA warps, the others group B's with GB warps;
// the warps a plan does not use leave at once.  Per tile the arithmetic is
// that of k_step_f32, so every problem gives the same bits as in its own
// group's launch.
template <bool PER, int DA, int ZA, int DB, int ZB, int R, int MAXT, int REGS>
__global__ void __launch_bounds__(MAXT) __maxnreg__(REGS)
k_step_f32_pair(const __grid_constant__ CUtensorMap unused, const __grid_constant__ ProblemDesc none,
                const ProblemDesc* __restrict__ table_a, int nprob_a, int ntiles_a, int ga,
                int ctas_a, const ProblemDesc* __restrict__ table_b, int nprob_b, int ntiles_b,
                int gb, unsigned* err, const DirTable ta, const DirTable tb) {
  if ((int)blockIdx.x < ctas_a) {
    if ((int)threadIdx.y >= ga) return;
    step_f32_body<1, PER, DA, ZA, R, true, !PER, false>(unused, none, table_a, nprob_a, ntiles_a, err, ta,
                                           blockIdx.x, ctas_a, ga);
  } else {
    if ((int)threadIdx.y >= gb) return;
    step_f32_body<1, PER, DB, ZB, R, true, !PER, false>(unused, none, table_b, nprob_b, ntiles_b, err, tb,
                                           blockIdx.x - ctas_a, gridDim.x - ctas_a, gb);
  }
}

template <int DPT, int ZC, int R>
size_t step_smem(int G) {
  return sizeof(float) * ((size_t)G * R * slot_floats<DPT, ZC>() + ZC * 5 * 64) +
         sizeof(DirConst) * (size_t)G * DPT + 8 * (size_t)G * R + sizeof(double) * 4 * ZC + 16;
}

template <int MODE, bool PER, int DPT, int ZC, int R, int MAXT, int REGS>
cudaError_t set_smem_attr() {
  // the opt-in shared-memory size is a per-device function attribute
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && (attr_set >> dev & 1ull)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(k_step_f32<MODE, PER, DPT, ZC, R, MAXT, REGS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024 - 1024);
  if (e == cudaSuccess && dev < 64) attr_set |= 1ull << dev;
  return e;
}

// Resident CTAs per SM; the two boundary specialisations have the same
// launch bounds and shared memory, the smaller count is returned.
template <int MODE, int DPT, int ZC, int R, int MAXT, int REGS>
cudaError_t occupancy_mode(int G, int* per_sm) {
  int a = 0, b = 0;
  cudaError_t e = set_smem_attr<MODE, false, DPT, ZC, R, MAXT, REGS>();
  if (e == cudaSuccess) e = set_smem_attr<MODE, true, DPT, ZC, R, MAXT, REGS>();
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &a, k_step_f32<MODE, false, DPT, ZC, R, MAXT, REGS>, 32 * G, step_smem<DPT, ZC, R>(G));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &b, k_step_f32<MODE, true, DPT, ZC, R, MAXT, REGS>, 32 * G, step_smem<DPT, ZC, R>(G));
  *per_sm = std::min(a, b);
  return e;
}

// the single-problem grid serves both the plain and the moments variant
template <bool BATCH, int DPT, int ZC, int R, int MAXT, int REGS>
cudaError_t occupancy(int G, int* per_sm) {
  if (BATCH) return occupancy_mode<1, DPT, ZC, R, MAXT, REGS>(G, per_sm);
  int a = 0, b = 0;
  cudaError_t e = occupancy_mode<0, DPT, ZC, R, MAXT, REGS>(G, &a);
  if (e == cudaSuccess) e = occupancy_mode<2, DPT, ZC, R, MAXT, REGS>(G, &b);
  *per_sm = std::min(a, b);
  return e;
}

bool any_periodic(const Grid& g) { return g.periodic[0] || g.periodic[1] || g.periodic[2]; }

template <int DPT, int ZC, int R, int MAXT, int REGS>
cudaError_t launch_f32(const StepLaunch& L, const StaticCoef& c, const DirTable& t,
                       cudaStream_t s, int* nblocks) {
  const int G = L.N / DPT;  // internal (padded) direction count / directions per warp
  if (!L.tmap_in || G < 1 || G * DPT != L.N || 32 * G > MAXT || L.nzc < 1 || L.nzc > L.g.nz ||
      L.ctas < 1)
    return cudaErrorInvalidValue;
  if (L.budget_partials && L.ctas > L.partials_cap) return cudaErrorInvalidValue;
  if (nblocks) *nblocks = L.ctas;
  const size_t smem = step_smem<DPT, ZC, R>(G);
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  const bool per = any_periodic(L.g);
  const bool mom = L.mom_E || L.mom_F;
  const cudaError_t e = mom ? (per ? set_smem_attr<2, true, DPT, ZC, R, MAXT, REGS>()
                                   : set_smem_attr<2, false, DPT, ZC, R, MAXT, REGS>())
                            : (per ? set_smem_attr<0, true, DPT, ZC, R, MAXT, REGS>()
                                   : set_smem_attr<0, false, DPT, ZC, R, MAXT, REGS>());
  if (e != cudaSuccess) return e;
  ProblemDesc one{};
  one.g = L.g;
  one.out = L.out;
  one.tmap = nullptr;
  one.cf = c;
  one.dt = L.dt;
  one.collision = L.collision;
  one.lambda_iters = L.lambda_iters;
  one.nzc = L.nzc;
  one.tile_start = 0;
  one.ntiles = (L.g.nx + 63) / 64 * L.g.ny * L.nzc;
  one.budget_partials = L.budget_partials;
  one.mom_E = L.mom_E;
  one.mom_F = L.mom_F;
  if (mom && per)
    k_step_f32<2, true, DPT, ZC, R, MAXT, REGS>
        <<<L.ctas, dim3(32, G), smem, s>>>(*L.tmap_in, one, nullptr, 1, one.ntiles, L.err, t);
  else if (mom)
    k_step_f32<2, false, DPT, ZC, R, MAXT, REGS>
        <<<L.ctas, dim3(32, G), smem, s>>>(*L.tmap_in, one, nullptr, 1, one.ntiles, L.err, t);
  else if (per)
    k_step_f32<0, true, DPT, ZC, R, MAXT, REGS>
        <<<L.ctas, dim3(32, G), smem, s>>>(*L.tmap_in, one, nullptr, 1, one.ntiles, L.err, t);
  else
    k_step_f32<0, false, DPT, ZC, R, MAXT, REGS>
        <<<L.ctas, dim3(32, G), smem, s>>>(*L.tmap_in, one, nullptr, 1, one.ntiles, L.err, t);
  return cudaGetLastError();
}

template <int DPT, int ZC, int R, int MAXT, int REGS>
cudaError_t launch_f32_batch(const BatchLaunch& B, const DirTable& t, cudaStream_t s) {
  const int G = B.N / DPT;
  if (G < 1 || G * DPT != B.N || 32 * G > MAXT || B.ctas < 1 || B.ntiles < 1 || !B.table ||
      B.nprob < 1)
    return cudaErrorInvalidValue;
  const size_t smem = step_smem<DPT, ZC, R>(G);
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  const cudaError_t e = B.periodic ? set_smem_attr<1, true, DPT, ZC, R, MAXT, REGS>()
                                   : set_smem_attr<1, false, DPT, ZC, R, MAXT, REGS>();
  if (e != cudaSuccess) return e;
  // the parameter-space tensor map and descriptor are unused by the batched kernel
  CUtensorMap unused{};
  ProblemDesc none{};
  if (B.periodic)
    k_step_f32<1, true, DPT, ZC, R, MAXT, REGS>
        <<<B.ctas, dim3(32, G), smem, s>>>(unused, none, B.table, B.nprob, B.ntiles, B.err, t);
  else
    k_step_f32<1, false, DPT, ZC, R, MAXT, REGS>
        <<<B.ctas, dim3(32, G), smem, s>>>(unused, none, B.table, B.nprob, B.ntiles, B.err, t);
  return cudaGetLastError();
}

constexpr int kRing = 2;

template <bool PER, int DA, int ZA, int DB, int ZB, int R, int MAXT, int REGS>
cudaError_t set_smem_attr_pair() {
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && (attr_set >> dev & 1ull)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(k_step_f32_pair<PER, DA, ZA, DB, ZB, R, MAXT, REGS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024 - 1024);
  if (e == cudaSuccess && dev < 64) attr_set |= 1ull << dev;
  return e;
}

template <int DA, int ZA, int DB, int ZB, int R>
size_t pair_smem(int ga, int gb) {
  return std::max(step_smem<DA, ZA, R>(ga), step_smem<DB, ZB, R>(gb));
}

template <int DA, int ZA, int DB, int ZB, int R, int MAXT, int REGS>
cudaError_t occupancy_pair(int ga, int gb, int* per_sm) {
  int a = 0, b = 0;
  const int threads = 32 * std::max(ga, gb);
  cudaError_t e = set_smem_attr_pair<false, DA, ZA, DB, ZB, R, MAXT, REGS>();
  if (e == cudaSuccess) e = set_smem_attr_pair<true, DA, ZA, DB, ZB, R, MAXT, REGS>();
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &a, k_step_f32_pair<false, DA, ZA, DB, ZB, R, MAXT, REGS>, threads,
        pair_smem<DA, ZA, DB, ZB, R>(ga, gb));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &b, k_step_f32_pair<true, DA, ZA, DB, ZB, R, MAXT, REGS>, threads,
        pair_smem<DA, ZA, DB, ZB, R>(ga, gb));
  *per_sm = std::min(a, b);
  return e;
}

template <int DA, int ZA, int DB, int ZB, int R, int MAXT, int REGS>
cudaError_t launch_f32_pair(const BatchLaunch& A, const DirTable& ta, const BatchLaunch& B,
                            const DirTable& tb, int ctas_a, int ctas, cudaStream_t s) {
  const int ga = A.N / DA, gb = B.N / DB;
  if (ga < 1 || ga * DA != A.N || gb < 1 || gb * DB != B.N || 32 * std::max(ga, gb) > MAXT ||
      ctas_a < 1 || ctas_a >= ctas || !A.table || !B.table || A.nprob < 1 || B.nprob < 1 ||
      A.ntiles < 1 || B.ntiles < 1)
    return cudaErrorInvalidValue;
  const size_t smem = pair_smem<DA, ZA, DB, ZB, R>(ga, gb);
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  const bool per = A.periodic || B.periodic;
  const cudaError_t e = per ? set_smem_attr_pair<true, DA, ZA, DB, ZB, R, MAXT, REGS>()
                            : set_smem_attr_pair<false, DA, ZA, DB, ZB, R, MAXT, REGS>();
  if (e != cudaSuccess) return e;
  CUtensorMap unused{};
  ProblemDesc none{};
  const dim3 block(32, std::max(ga, gb));
  if (per)
    k_step_f32_pair<true, DA, ZA, DB, ZB, R, MAXT, REGS><<<ctas, block, smem, s>>>(
        unused, none, A.table, A.nprob, A.ntiles, ga, ctas_a, B.table, B.nprob, B.ntiles, gb,
        B.err, ta, tb);
  else
    k_step_f32_pair<false, DA, ZA, DB, ZB, R, MAXT, REGS><<<ctas, block, smem, s>>>(
        unused, none, A.table, A.nprob, A.ntiles, ga, ctas_a, B.table, B.nprob, B.ntiles, gb,
        B.err, ta, tb);
  return cudaGetLastError();
}


// Dispatch over the compiled tile plans (directions per warp, planes per
// batch, thread cap, registers per thread), in order of preference.  A
// scheduler holds floor(16384 / (32 x registers)) warps: 96 registers allow
// 5 warps per scheduler (two CTAs of 9 warps, ico42 with 45 internal
// directions, or one of 17), 128 allow 4 (one CTA of 16 warps: ico162 with 176
// internal directions at 11 per warp).
#define LBRT_TILE_PLANS(X) \
  X(5, 2, 320, 96)         \
  X(11, 1, 512, 128)       \
  X(10, 1, 544, 96)        \
  X(8, 2, 512, 128)        \
  X(4, 2, 512, 128)        \
  X(4, 1, 640, 96)

}  // namespace

// Alternative batched kernels (directions per warp, planes per batch, thread
// cap, registers) with the memory layout of the tile plan of the same
// directions per warp: the batch autotuner times them against the plan's
// own kernel.  One plane per batch at 72 registers holds three 9-warp CTAs
// per SM instead of two.
#define LBRT_BATCH_ALT(X) X(5, 1, 320, 72)

// Plan pairs that share one batched launch (plan A, plan B, thread cap,
// registers): the 42-direction (5 per warp, 2 planes) and the 162-direction
// (11 per warp) icosahedral sets.
#define LBRT_PAIR_PLANS(X) X(5, 2, 11, 1, 512, 128)

#define LBRT_PLAN_ROW(D, Z, T, B) {D, Z, T},
const int kTilePlans[][3] = {LBRT_TILE_PLANS(LBRT_PLAN_ROW)};
#undef LBRT_PLAN_ROW
const int kNumTilePlans = sizeof(kTilePlans) / sizeof(kTilePlans[0]);

size_t step_tile_smem(int dpt, int zc, int warps) {
#define LBRT_SMEM(D, Z, T, B) \
  if (dpt == D && zc == Z) return step_smem<D, Z, kRing>(warps);
  LBRT_TILE_PLANS(LBRT_SMEM)
#undef LBRT_SMEM
  return (size_t)-1;
}

int batch_alt_zc(int storage, int dpt) {
  if (storage != ST_F32) return batch_alt_zc16(dpt);
#define LBRT_AZ(D, Z, T, R_) \
  if (dpt == D) return Z;
  LBRT_BATCH_ALT(LBRT_AZ)
#undef LBRT_AZ
  return 0;
}

cudaError_t launch_tma_static_batch(const BatchLaunch& B, const DirTable& t, cudaStream_t s) {
  if (B.storage != ST_F32) return launch_tma16_static_batch(B, t, s);
  if (B.alt) {
#define LBRT_LAUNCHA(D, Z, T, R_) \
  if (B.dpt == D && B.zc == Z) return launch_f32_batch<D, Z, kRing, T, R_>(B, t, s);
    LBRT_BATCH_ALT(LBRT_LAUNCHA)
#undef LBRT_LAUNCHA
    return cudaErrorInvalidValue;
  }
#define LBRT_LAUNCHB(D, Z, T, R_) \
  if (B.dpt == D && B.zc == Z) return launch_f32_batch<D, Z, kRing, T, R_>(B, t, s);
  LBRT_TILE_PLANS(LBRT_LAUNCHB)
#undef LBRT_LAUNCHB
  return cudaErrorInvalidValue;
}

cudaError_t occupancy_static_batch(int storage, int dpt, int zc, int G, int* per_sm, int alt) {
  if (storage != ST_F32) return occupancy_tma16(storage, dpt, zc, G, per_sm, true, alt);
  cudaError_t e = cudaErrorInvalidValue;
  if (alt) {
#define LBRT_OCCA(D, Z, T, R_) \
  if (dpt == D && zc == Z) e = occupancy<true, D, Z, kRing, T, R_>(G, per_sm);
    LBRT_BATCH_ALT(LBRT_OCCA)
#undef LBRT_OCCA
    return e;
  }
#define LBRT_OCCB(D, Z, T, R_) \
  if (dpt == D && zc == Z) e = occupancy<true, D, Z, kRing, T, R_>(G, per_sm);
  LBRT_TILE_PLANS(LBRT_OCCB)
#undef LBRT_OCCB
  return e;
}

bool static_batch_pair_supported(int storage, int dpt_a, int zc_a, int dpt_b, int zc_b) {
  if (storage != ST_F32) return tma16_pair_supported(dpt_a, zc_a, dpt_b, zc_b);
#define LBRT_PS(DA, ZA, DB, ZB, T, R_) \
  if (dpt_a == DA && zc_a == ZA && dpt_b == DB && zc_b == ZB) return true;
  LBRT_PAIR_PLANS(LBRT_PS)
#undef LBRT_PS
  return false;
}

cudaError_t launch_static_batch_pair(const BatchLaunch& A, const DirTable& ta, const BatchLaunch& B,
                                     const DirTable& tb, int ctas_a, int ctas, cudaStream_t s) {
  if (A.storage != B.storage) return cudaErrorInvalidValue;
  if (A.storage != ST_F32) return launch_tma16_static_batch_pair(A, ta, B, tb, ctas_a, ctas, s);
#define LBRT_LP(DA, ZA, DB, ZB, T, R_)                                                    \
  if (A.dpt == DA && A.zc == ZA && B.dpt == DB && B.zc == ZB)                            \
    return launch_f32_pair<DA, ZA, DB, ZB, kRing, T, R_>(A, ta, B, tb, ctas_a, ctas, s);
  LBRT_PAIR_PLANS(LBRT_LP)
#undef LBRT_LP
  return cudaErrorInvalidValue;
}

cudaError_t occupancy_static_batch_pair(int storage, int dpt_a, int zc_a, int ga, int dpt_b,
                                        int zc_b, int gb, int* per_sm) {
  if (storage != ST_F32)
    return occupancy_tma16_pair(storage, dpt_a, zc_a, ga, dpt_b, zc_b, gb, per_sm);
#define LBRT_OP(DA, ZA, DB, ZB, T, R_)                                                    \
  if (dpt_a == DA && zc_a == ZA && dpt_b == DB && zc_b == ZB)                            \
    return occupancy_pair<DA, ZA, DB, ZB, kRing, T, R_>(ga, gb, per_sm);
  LBRT_PAIR_PLANS(LBRT_OP)
#undef LBRT_OP
  return cudaErrorInvalidValue;
}

cudaError_t launch_tma_static(const StepLaunch& L, const StaticCoef& c, const DirTable& t,
                              int dpt, int zc, cudaStream_t s, int* nblocks) {
#define LBRT_LAUNCH(D, Z, T, B) \
  if (dpt == D && zc == Z) return launch_f32<D, Z, kRing, T, B>(L, c, t, s, nblocks);
  LBRT_TILE_PLANS(LBRT_LAUNCH)
#undef LBRT_LAUNCH
  return cudaErrorInvalidValue;
}

// Persistent grid of the static kernel: CTAs = resident CTAs per SM x SMs
// (at most one per tile), and the number of z chunks nzc that minimises the
// busiest CTA's share of plane loads under the round-robin tile order (each
// tile loads zlen + 1 planes rounded up to whole batches, plus a small
// per-tile overhead).
cudaError_t plan_static_grid(const Grid& g, int Ni, int dpt, int zc, int storage, int* nzc,
                             int* ctas, bool moving, bool sc) {
  const int G = Ni / dpt;
  int per_sm = 0;
  cudaError_t e = cudaErrorInvalidValue;
  if (sc) {
    e = occupancy_sc(storage, dpt, zc, G, &per_sm);
  } else if (moving) {
    e = storage == ST_F32 ? occupancy_tma_moving(dpt, G, &per_sm)
                          : occupancy_tma16_moving(storage, dpt, G, &per_sm);
  } else if (storage == ST_F32) {
#define LBRT_OCC(D, Z, T, B) \
  if (dpt == D && zc == Z) e = occupancy<false, D, Z, kRing, T, B>(G, &per_sm);
    LBRT_TILE_PLANS(LBRT_OCC)
#undef LBRT_OCC
  } else {
    e = occupancy_tma16(storage, dpt, zc, G, &per_sm);
  }
  if (e != cudaSuccess) return e;
  if (per_sm < 1) return cudaErrorInvalidConfiguration;
  int dev = 0, sms = 0;
  e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  if (e != cudaSuccess) return e;
  const long long slots = (long long)per_sm * sms;
  const int nxb = (g.nx + 63) / 64;
  const long long txy = (long long)nxb * g.ny;
  // With a periodic x axis the tiles of the first and last x-block also write
  // the ghost columns.  Tiles are numbered x-block fastest and CTA b takes
  // tiles b, b + C, ...: when C is a multiple of the x-blocks per row, every
  // CTA keeps one x-block and the ghost-writing CTAs fall behind the others
  // for the whole step.  A CTA count coprime to the x-blocks rotates every CTA
  // through all x-blocks (measured with two CTAs per SM, 256^3 x 42 periodic:
  // 2.09 -> 1.78 ms).  With one CTA per SM an idle SM costs more than it
  // saves; those grids keep every SM and the static kernels permute the
  // x-blocks of each round instead (tile_rot).
  const bool rotate = g.periodic[0] && per_sm >= 2 && nxb > 1;
  auto grid_ctas = [&](long long nt) {
    long long nc = std::min(nt, slots);
    if (rotate)
      while (nc > 1 && std::gcd(nc, (long long)nxb) > 1) --nc;
    return nc;
  };
  double best = 1e300;
  int best_c = 1;
  const int cmax = std::min(g.nz, 64);
  for (int c = 1; c <= cmax; ++c) {
    const long long nt = txy * c;
    if (nt > (1LL << 24)) break;
    const long long nc = grid_ctas(nt);
    const int base = g.nz / c, rem = g.nz % c;
    auto cost = [&](long long ti) {
      const long long ch = ti / txy;
      const int zlen = base + (ch < rem ? 1 : 0);
      return (double)((zlen + 1 + zc - 1) / zc * zc) + 0.5;
    };
    double worst = 0.0;  // the busiest CTA of the round-robin order
    for (long long b = 0; b < nc; ++b) {
      double sum = 0.0;
      for (long long ti = b; ti < nt; ti += nc) sum += cost(ti);
      worst = std::max(worst, sum);
    }
    if (worst < best * 0.999) {
      best = worst;
      best_c = c;
    }
  }
  *nzc = best_c;
  *ctas = (int)grid_ctas(txy * best_c);
  return cudaSuccess;
}

PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder(std::string& err) {
  static PFN_cuTensorMapEncodeTiled_v12000 encode = nullptr;
  if (!encode) {
    cudaDriverEntryPointQueryResult q;
    void* fn = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &fn, 12000, cudaEnableDefault,
                                         &q) != cudaSuccess ||
        q != cudaDriverEntryPointSuccess || !fn) {
      err = "cuTensorMapEncodeTiled is not available from the driver";
      return nullptr;
    }
    encode = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(fn);
  }
  return encode;
}

bool make_pop_tensor_map(CUtensorMap* map, const Grid& g, int Ni, void* base, int dpt, int zc,
                         std::string& err) {
  auto encode = tensor_map_encoder(err);
  if (!encode) return false;
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
