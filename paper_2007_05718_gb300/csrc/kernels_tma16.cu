// Fused stream + collide step for a static fluid with 16-bit (FP16 or BF16)
// population storage, fed by TMA tensor tiles.  Weih et al. 2020: Sec. 3.3,
// Eqs. (interp), (rte_implicit), (collision-step); the storage format is this
// library's own (the paper keeps populations in double precision).
//
// Storage.  Per site the energy density E is kept in float32 (padded array
// [PZ][PY][PX], same ghost layer and periodic mirrors as the populations),
// and per site and direction the relative deviation from the static local
// equilibrium I_i = w_i E is kept in 16 bits:
//   f_i = I_i / w_i = E^ (1 + q_i),   E^ = max(E, 1e-30).
// q_i is bounded by the direction count (I_i <= E), so it fits the 16-bit
// range without a scale, and its rounding error is relative to the
// deviation, not to I_i.  All arithmetic is float32: the stream works on
// f_i (the weight w_i is constant along a direction and factors out of Eq.
// (interp)), moments use the pairs (w_i, w_i n_i), and the output is encoded
// directly as q_i = (A / E^') f*_i + (c0 / E^' - 1) + n_i . (c1 / E^') with
// E^' the site's new energy density.
//
// Work decomposition, data movement and the tile schedule are those of the
// float32 kernel (kernels_tma.cu): per batch a warp loads one box of its
// DPT directions x 2 rows x ZC planes x 72 columns, and the CTA loads one box
// of E over the three rows y - 1 .. y + 1 and ZC + 1 planes, shared by all
// warps.
#include <algorithm>

#include "lb_rt_internal.h"
#include "tma_common.cuh"

#include <cudaTypedefs.h>

namespace lbrt {

namespace {

using namespace tma;

constexpr int BOXH = 72;  // 16-bit columns per box row: sites x0 - 2 .. x0 + 69
constexpr float EPS_E = 1e-30f;

template <class ST> struct Conv;
template <> struct Conv<__half> {
  using T2 = __half2;
  static __device__ __forceinline__ float2 to2(T2 v) { return __half22float2(v); }
  static __device__ __forceinline__ float to1(__half v) { return __half2float(v); }
  static __device__ __forceinline__ T2 from2(float2 v) { return __float22half2_rn(v); }
};
template <> struct Conv<__nv_bfloat16> {
  using T2 = __nv_bfloat162;
  static __device__ __forceinline__ float2 to2(T2 v) { return __bfloat1622float2(v); }
  static __device__ __forceinline__ float to1(__nv_bfloat16 v) { return __bfloat162float(v); }
  static __device__ __forceinline__ T2 from2(float2 v) { return __float22bfloat162_rn(v); }
};

// Per-direction constants (pre-broadcast pairs): s0 = (a_x, a_x, a_y, a_y),
// s1 = (a_z', a_z', n_x, n_x), s2 = (n_y, n_y, n_z, n_z), m0 = (w, w, w n_x,
// w n_x), m1 = (w n_y, w n_y, w n_z, w n_z); sh = -1 when the x-upwind
// neighbour is x - 1 (sgn n^x = +1), +1 otherwise.
struct DirConst16 {
  float4 s0, s1, s2, m0, m1;
  int sh, inert, pad0, pad1;
};

template <int DPT, int ZC>
__host__ __device__ constexpr int slot_bytes16() {
  return ((BOXH * DPT * 2 * ZC * 2 + 127) / 128) * 128;
}
template <int ZC>
__host__ __device__ constexpr int eslot_floats() {
  return ((BOXH * 3 * (ZC + 1) * 4 + 127) / 128) * 32;
}

// Store a float32 site value into the padded E array and every periodic
// ghost mirror of the site.
__device__ __forceinline__ void store_e(float* e, const Grid& g, int z, int y, int x, float v) {
  int xs[3], ys[3], zs[3];
  const int nxs = mirrors(x, g.nx, g.periodic[0], GL, xs);
  const int nys = mirrors(y, g.ny, g.periodic[1], 1, ys);
  const int nzs = mirrors(z, g.nz, g.periodic[2], 1, zs);
  const long long ey = g.PX, ez = (long long)g.PX * g.PY;
  for (int a = 0; a < nzs; ++a)
    for (int b = 0; b < nys; ++b)
      for (int c = 0; c < nxs; ++c) e[zs[a] * ez + ys[b] * ey + xs[c]] = v;
}

// BATCH as in the float32 kernel: one problem in the parameter space, or a
// device array of problem descriptors walked by the persistent CTAs.
// PER as in the float32 kernel: periodic axes take the fast store path
// that also writes ghost columns and mirror rows / planes.
// The body runs on CTA `cta` of `ncta` persistent CTAs with G warps; PART:
// the block belongs to a launch shared by two tile plans (k_step_16_pair).
// ROT: permute the x-blocks of each round of tiles (tile_rot), compiled in for
// the single-problem plans of one CTA per SM.
template <class ST, bool BATCH, bool PER, int DPT, int ZC, int R, bool PART, bool ROT>
__device__ __forceinline__ void step16_body(const CUtensorMap& tmap1, const CUtensorMap& emap1,
                                            const ProblemDesc& one,
                                            const ProblemDesc* __restrict__ table, int nprob,
                                            int ntiles, unsigned* err, const DirTable& t,
                                            const int cta, const int ncta, const int G) {
  using C2 = Conv<ST>;
  using T2 = typename C2::T2;
  constexpr int SLOTB = slot_bytes16<DPT, ZC>();
  constexpr int ESLOT = eslot_floats<ZC>();
  static_assert(SLOTB >= ZC * 4 * 64 * 4, "the partial moments must fit in a consumed slot");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int lane = threadIdx.x, g = threadIdx.y;
  __shared__ ProblemDesc pd[BATCH ? 2 : 1];
  // shared layout: ring [G][R][SLOTB] | E ring [R][ESLOT] | coef [ZC][5][64] |
  // dirs [N] | mbar [G][R] | ebar [R] | budget [2 ZC][2] double | abort flag
  unsigned char* ring = smem_raw;
  float* ering = reinterpret_cast<float*>(ring + (size_t)G * R * SLOTB);
  float* coef = ering + R * ESLOT;
  DirConst16* dirs = reinterpret_cast<DirConst16*>(coef + ZC * 5 * 64);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(dirs + G * DPT);
  unsigned long long* ebar = mbar + G * R;
  double* bsum = reinterpret_cast<double*>(ebar + R);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bsum + 4 * ZC);

  const int i0 = g * DPT;
  const int oct0 = __float_as_int(t.au[i0].w);
  const bool yneg = oct0 & 2;
  const int zs = (oct0 & 4) ? 1 : 0;
  const int row_own = yneg ? 0 : 1, row_up = yneg ? 1 : 0;  // rows of a population box
  const int erow_up = yneg ? 2 : 0;                          // rows of the E box: y-1, y, y+1
  const int nunits = 2 * ZC;

  for (int i = g * 32 + lane; i < G * DPT; i += G * 32) {
    const float4 au = t.au[i], nw = t.nw[i];
    const int oct = __float_as_int(au.w);
    const float azw = (oct & 4) ? 1.f - au.z : au.z;
    DirConst16 d;
    d.s0 = make_float4(au.x, au.x, au.y, au.y);
    d.s1 = make_float4(azw, azw, nw.x, nw.x);
    d.s2 = make_float4(nw.y, nw.y, nw.z, nw.z);
    const float wx = nw.w * nw.x, wy = nw.w * nw.y, wz = nw.w * nw.z;
    d.m0 = make_float4(nw.w, nw.w, wx, wx);
    d.m1 = make_float4(wy, wy, wz, wz);
    d.sh = (oct & 1) ? 1 : -1;
    d.inert = oct & 8;
    d.pad0 = d.pad1 = 0;
    dirs[i] = d;
  }
  if (lane == 0) {
    for (int r = 0; r < R; ++r) mbar_init(smem_u32(&mbar[g * R + r]), 1);
    if (g == 0)
      for (int r = 0; r < R; ++r) mbar_init(smem_u32(&ebar[r]), 1);
  }
  if (g == 0 && lane == 0) *abort_flag = 0;
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  cta_sync<PART>(32 * G);
  unsigned inert_mask = 0;
#pragma unroll
  for (int k = 0; k < DPT; ++k) inert_mask |= dirs[i0 + k].inert ? 1u << k : 0u;

  unsigned char* my_ring = ring + (size_t)g * R * SLOTB;
  bool alive = true;
  int issued = 0, waited = 0;
  int is_t = cta, is_p = 0, is_m = 0, is_M = 0, is_x0 = 0, is_yp = 0, is_zp = 0, is_y = 0,
      is_zb = 0;
  const CUtensorMap* is_map = &tmap1;
  const CUtensorMap* is_emap = &emap1;
  auto issue_seek = [&]() {
    if (is_t < ntiles) {
      if constexpr (BATCH) {
        while (is_p < nprob && is_t >= table[is_p].tile_start + table[is_p].ntiles) ++is_p;
        if (is_p >= nprob) {  // inconsistent table: stop issuing (the consumer reports it)
          is_t = ntiles;
          return;
        }
        is_map = table[is_p].tmap;
        is_emap = table[is_p].emap;
      }
      const ProblemDesc& D = BATCH ? table[is_p] : one;
      const int nxb_i = (D.g.nx + 63) / 64, rel_i = is_t - D.tile_start;
      const TileGeom tg = tile_geom(rel_i, nxb_i, D.g.ny, D.g.nz, D.nzc,
                                    ROT ? tile_rot(rel_i, nxb_i, ncta, D.g.periodic[0]) : 0);
      is_M = tile_items<ZC>(tg.zlen);
      is_x0 = tg.x0;
      is_y = tg.y;
      is_yp = yneg ? tg.y + 1 : tg.y;
      is_zb = tg.zbeg;
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
      mbar_arrive_tx(bar, BOXH * DPT * 2 * ZC * 2);
      tma_load_4d(smem_u32(my_ring + (size_t)slot * SLOTB), is_map, is_x0, i0, is_yp,
                  is_zp + is_m * ZC, bar);
      if (g == 0) {
        const uint32_t eb = smem_u32(&ebar[slot]);
        mbar_arrive_tx(eb, BOXH * 3 * (ZC + 1) * 4);
        tma_load_3d(smem_u32(ering + (size_t)slot * ESLOT), is_emap, is_x0, is_y,
                    is_zb + is_m * ZC, eb);
      }
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
    const uint32_t par = (uint32_t)((q / R) & 1);
    if (!mbar_wait(smem_u32(&mbar[g * R + q % R]), par, err) ||
        !mbar_wait(smem_u32(&ebar[q % R]), par, err)) {
      *abort_flag = 1;
      alive = false;
      return false;
    }
    waited = q + 1;
    return true;
  };
  const int wc = 2 + 2 * lane;  // window column of the lane's pair

  while (issued < R - 1 && issue()) {
  }

  float2 carry[DPT];
#pragma unroll
  for (int k = 0; k < DPT; ++k) carry[k] = make_float2(0.f, 0.f);
  float bud_a = 0.f, bud_b = 0.f;
  double bud_da = 0.0, bud_db = 0.0;
  int q = 0;
  int tk = 0;
  int cp = 0;
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
    ST* __restrict__ out = static_cast<ST*>(P.out);
    float* __restrict__ eout = P.e_out;
    const StaticCoef& cf = P.cf;
    const int nxb_t = (nx + 63) / 64, rel_t = ti - P.tile_start;
    const TileGeom tg = tile_geom(rel_t, nxb_t, ny, nz, P.nzc,
                                  ROT ? tile_rot(rel_t, nxb_t, ncta, gr.periodic[0]) : 0);
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
    ST* const orow = out + (long long)i0 * gr.si + (long long)(y + 1) * gr.sy + xa + GL;
    for (int m = 0; m < M; ++m, ++q) {
      const int zb = zbeg - 1 + m * ZC;
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
      wait_item(q);
      unsigned char* slot = my_ring + (size_t)(q % R) * SLOTB;
      const ST* sl = reinterpret_cast<const ST*>(slot);
      const float* es = ering + (size_t)(q % R) * ESLOT;
      // E^ of the lane's pair and of the two x-neighbours, own and upwind row
      float2 EPo[ZC], EPu[ZC];
      float Emo[ZC], Epo[ZC], Emu[ZC], Epu[ZC];
#pragma unroll
      for (int j = 0; j < ZC; ++j) {
        const float* eo = es + ((j + zs) * 3 + 1) * BOXH + wc;
        const float* eu = es + ((j + zs) * 3 + erow_up) * BOXH + wc;
        EPo[j] = *reinterpret_cast<const float2*>(eo);
        EPu[j] = *reinterpret_cast<const float2*>(eu);
        Emo[j] = eo[-1];
        Epo[j] = eo[2];
        Emu[j] = eu[-1];
        Epu[j] = eu[2];
      }
      float2 Is[DPT][ZC];
      float2 aE[ZC], aX[ZC], aY[ZC], aZ[ZC];
#pragma unroll
      for (int j = 0; j < ZC; ++j) aE[j] = aX[j] = aY[j] = aZ[j] = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < DPT; ++k) {
        const DirConst16& d = dirs[i0 + k];
        const float4 s0 = d.s0, s1 = d.s1, m0 = d.m0, m1 = d.m1;
        const float2 ax = make_float2(s0.x, s0.y), ay = make_float2(s0.z, s0.w);
        const float2 az = make_float2(s1.x, s1.y);
        const float2 w2 = make_float2(m0.x, m0.y), wx2 = make_float2(m0.z, m0.w);
        const float2 wy2 = make_float2(m1.x, m1.y), wz2 = make_float2(m1.z, m1.w);
        // Eq. (interp) on the decoded f = E^ (1 + q): x on both rows, then y,
        // then z against the carried plane; the x-upwind neighbour decides
        // which edge value completes the shifted pair
        auto pass = [&](auto xneg) {
#pragma unroll
          for (int j = 0; j < ZC; ++j) {
            const ST* po = sl + ((j * 2 + row_own) * DPT + k) * BOXH + wc;
            const ST* pu = sl + ((j * 2 + row_up) * DPT + k) * BOXH + wc;
            const float2 qo = C2::to2(*reinterpret_cast<const T2*>(po));
            const float2 qu = C2::to2(*reinterpret_cast<const T2*>(pu));
            const float2 fo = f2fma(EPo[j], qo, EPo[j]);
            const float2 fu = f2fma(EPu[j], qu, EPu[j]);
            float2 So, Su;
            if (decltype(xneg)::value) {
              const float eo = fmaf(Epo[j], C2::to1(po[2]), Epo[j]);
              const float eu = fmaf(Epu[j], C2::to1(pu[2]), Epu[j]);
              So = make_float2(fo.y, eo);
              Su = make_float2(fu.y, eu);
            } else {
              const float eo = fmaf(Emo[j], C2::to1(po[-1]), Emo[j]);
              const float eu = fmaf(Emu[j], C2::to1(pu[-1]), Emu[j]);
              So = make_float2(eo, fo.x);
              Su = make_float2(eu, fu.x);
            }
            const float2 X0 = f2fma(ax, f2sub(So, fo), fo);
            const float2 X1 = f2fma(ax, f2sub(Su, fu), fu);
            const float2 Bn = f2fma(ay, f2sub(X1, X0), X0);
            const float2 r = f2fma(az, f2sub(carry[k], Bn), Bn);
            carry[k] = Bn;
            Is[k][j] = r;
            aE[j] = f2fma(w2, r, aE[j]);
            aX[j] = f2fma(wx2, r, aX[j]);
            aY[j] = f2fma(wy2, r, aY[j]);
            aZ[j] = f2fma(wz2, r, aZ[j]);
          }
        };
        if (d.sh > 0) pass(std::true_type());
        else pass(std::false_type());
      }
      __syncwarp();
#pragma unroll
      for (int j = 0; j < ZC; ++j) {
        float2* p = reinterpret_cast<float2*>(slot + j * 4 * 64 * 4) + lane;
        p[0] = aE[j];
        p[32] = aX[j];
        p[64] = aY[j];
        p[96] = aZ[j];
      }
      cta_sync<PART>(32 * G);
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
          const float* p =
              reinterpret_cast<const float*>(ring + ((size_t)qq * R + s) * SLOTB) + j * 4 * 64 + f;
          E += p[0];
          Fx += p[64];
          Fy += p[128];
          Fz += p[192];
        }
        const Coef cc =
            collide_scalars(P.collision, P.lambda_iters, P.dt, inv_d, ka, k0, lam, eta, E, Fx, Fy, Fz);
        // q' = f' / E^' - 1 with E^' = max(E', eps): the coefficients of the
        // float32 path scaled by 1 / E^'
        const float Eh = fmaxf(cc.Enew, EPS_E);
        const float ri = __fdividef(1.f, Eh);
        float* c = coef + j * 5 * 64 + f;
        c[0] = cc.alpha * ri;
        c[64] = fmaf(cc.c0, ri, -1.f);
        c[128] = cc.c1x * ri;
        c[192] = cc.c1y * ri;
        c[256] = cc.c1z * ri;
        if (v) {
          bud_a += E;
          bud_b += cc.Enew;
          if (alive) store_e(eout, gr, z, y, x, Eh);
        }
      }
      cta_sync<PART>(32 * G);
      if (!BATCH && one.budget_partials && g < nunits) {
        bud_da += (double)bud_a;
        bud_db += (double)bud_b;
        bud_a = bud_b = 0.f;
      }
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
      // a warp with a lane on a periodic x edge also writes the x ghost column
      const bool fast = __all_sync(0xffffffffu, in0 && in1) && batch_plain;
      const bool xghost = __any_sync(0xffffffffu, gx_lo || gx_hi);
      bool done_fast = false;
      if constexpr (!PER) {
        if (alive && fast) {
          ST* base = orow + (long long)(zb + 1) * gr.sz;
#pragma unroll
          for (int k = 0; k < DPT; ++k) {
            if (inert_mask >> k & 1u) continue;
            const DirConst16& d = dirs[i0 + k];
            const float4 s1 = d.s1, s2 = d.s2;
            const float2 nx2 = make_float2(s1.z, s1.w);
            const float2 ny2 = make_float2(s2.x, s2.y), nz2 = make_float2(s2.z, s2.w);
#pragma unroll
            for (int j = 0; j < ZC; ++j) {
              const float2 qn =
                  f2fma(al[j], Is[k][j], f2fma(nz2, c1z[j], f2fma(ny2, c1y[j], f2fma(nx2, c1x[j], c0[j]))));
              *reinterpret_cast<T2*>(base + (long long)k * gr.si + (long long)j * gr.sz) = C2::from2(qn);
            }
          }
          done_fast = true;
        }
      } else {
        if (alive && fast) {
          ST* base = orow + (long long)(zb + 1) * gr.sz;
#pragma unroll
          for (int k = 0; k < DPT; ++k) {
            if (inert_mask >> k & 1u) continue;
            const DirConst16& d = dirs[i0 + k];
            const float4 s1 = d.s1, s2 = d.s2;
            const float2 nx2 = make_float2(s1.z, s1.w);
            const float2 ny2 = make_float2(s2.x, s2.y), nz2 = make_float2(s2.z, s2.w);
#pragma unroll
            for (int j = 0; j < ZC; ++j) {
              const float2 qn =
                  f2fma(al[j], Is[k][j], f2fma(nz2, c1z[j], f2fma(ny2, c1y[j], f2fma(nx2, c1x[j], c0[j]))));
              ST* dst = base + (long long)k * gr.si + (long long)j * gr.sz;
              const T2 h = C2::from2(qn);
              auto put = [&](ST* d) {
                *reinterpret_cast<T2*>(d) = h;
                if (xghost && gx_any) d[gx_off] = gx_y ? h.y : h.x;  // one predicated store
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
          const DirConst16& d = dirs[i0 + k];
          const float4 s1 = d.s1, s2 = d.s2;
          const float2 nx2 = make_float2(s1.z, s1.w);
          const float2 ny2 = make_float2(s2.x, s2.y), nz2 = make_float2(s2.z, s2.w);
#pragma unroll
          for (int j = 0; j < ZC; ++j) {
            if (!zok[j]) continue;
            const int z = zb + j;
            const float2 qn =
                f2fma(al[j], Is[k][j], f2fma(nz2, c1z[j], f2fma(ny2, c1y[j], f2fma(nx2, c1x[j], c0[j]))));
            const T2 h = C2::from2(qn);
            const ST hx = h.x, hy = h.y;
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
      }
    }
  }
  for (int qq = waited; qq < issued; ++qq) {
    const uint32_t par = (uint32_t)((qq / R) & 1);
    mbar_wait(smem_u32(&mbar[g * R + qq % R]), par, err);
    if (g == 0) mbar_wait(smem_u32(&ebar[qq % R]), par, err);
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

template <class ST, bool BATCH, bool PER, int DPT, int ZC, int R, int MAXT, int REGS>
__global__ void __launch_bounds__(MAXT) __maxnreg__(REGS)
k_step_16(const __grid_constant__ CUtensorMap tmap1, const __grid_constant__ CUtensorMap emap1,
          const __grid_constant__ ProblemDesc one, const ProblemDesc* __restrict__ table,
          int nprob, int ntiles, unsigned* err, const DirTable t) {
  constexpr bool ROT = PER && !BATCH && 2 * MAXT * REGS > 65536;
  step16_body<ST, BATCH, PER, DPT, ZC, R, false, ROT>(tmap1, emap1, one, table, nprob, ntiles, err,
                                                      t, blockIdx.x, gridDim.x, blockDim.y);
}

// One batched launch over the problems of two groups with different tile
// plans (for instance the 42- and the 162-direction icosahedral sets): CTAs
// 0 .. ctas_a - 1 walk group A's tiles with GA warps, the others group B's
// with GB warps.  The block has max(GA, GB) warps; the warps a plan does not
// use leave at once.  Per tile the arithmetic is that of k_step_16, so every
// problem gives the same bits as in its own group's launch.
template <class ST, bool PER, int DA, int ZA, int DB, int ZB, int R, int MAXT, int REGS>
__global__ void __launch_bounds__(MAXT) __maxnreg__(REGS)
k_step_16_pair(const __grid_constant__ CUtensorMap unused, const __grid_constant__ ProblemDesc none,
               const ProblemDesc* __restrict__ table_a, int nprob_a, int ntiles_a, int ga,
               int ctas_a, const ProblemDesc* __restrict__ table_b, int nprob_b, int ntiles_b,
               int gb, unsigned* err, const DirTable ta, const DirTable tb) {
  if ((int)blockIdx.x < ctas_a) {
    if ((int)threadIdx.y >= ga) return;
    step16_body<ST, true, PER, DA, ZA, R, true, false>(unused, unused, none, table_a, nprob_a, ntiles_a,
                                                err, ta, blockIdx.x, ctas_a, ga);
  } else {
    if ((int)threadIdx.y >= gb) return;
    step16_body<ST, true, PER, DB, ZB, R, true, false>(unused, unused, none, table_b, nprob_b, ntiles_b,
                                                err, tb, blockIdx.x - ctas_a, gridDim.x - ctas_a,
                                                gb);
  }
}

// Moving background fluid (App. B) with 16-bit storage: the tiled moving
// step of kernels_tma_moving.cu written in f = I / w.  With g'_i = A_i dt
// (W beta_i)^-3 (so g_i = w_i g'_i), the warps accumulate sum w f*,
// X = sum w beta^2 (g' eta_t + A f*), Y = sum w beta^2 g', sum w A f* and
// sum w g'; the units form src = eta_t + kt_0 J and E' = sum w A f* + src
// sum w g', store E^' and hand (src, 1/E^') to the output, which encodes
// q = (A f* + g' src) / E^' - 1.  One plane per batch.
struct DirConstM16 {
  float4 s0, s1, s2, s3;  // (a_x, a_y), (a_z', n_x), (n_y, n_z), (w, dt) pairs
  int sh, inert, pad0, pad1;
};

template <class ST, bool PER, int DPT, int R, int MAXT, int REGS>
__global__ void __launch_bounds__(MAXT) __maxnreg__(REGS)
k_step_moving16(const __grid_constant__ CUtensorMap tmap, const __grid_constant__ CUtensorMap emap,
                const StepLaunch L, const MovingCoef mc, const DirTable t) {
  using C2 = Conv<ST>;
  using T2 = typename C2::T2;
  constexpr int ZC = 1;
  constexpr int SLOTB = slot_bytes16<DPT, ZC>();
  constexpr int ESLOT = eslot_floats<ZC>();
  static_assert(SLOTB >= 5 * 64 * 4, "the partial sums must fit in a consumed slot");
  extern __shared__ __align__(128) unsigned char smem_raw[];
  const int G = blockDim.y;
  const int lane = threadIdx.x, g = threadIdx.y;
  const Grid& gr = L.g;
  const int nx = gr.nx, ny = gr.ny, nz = gr.nz;
  unsigned char* ring = smem_raw;
  float* ering = reinterpret_cast<float*>(ring + (size_t)G * R * SLOTB);
  float* coef = ering + R * ESLOT;  // [2][64]: src, 1 / E^'
  // per-site fields (vx, vy, vz, kt_a, kt_0, eta_t) of the current and the
  // next item, copied in by the last warp one item ahead
  float* fbuf = coef + 2 * 64;
  DirConstM16* dirs = reinterpret_cast<DirConstM16*>(fbuf + 2 * 6 * 64);
  unsigned long long* mbar = reinterpret_cast<unsigned long long*>(dirs + G * DPT);
  unsigned long long* ebar = mbar + G * R;
  double* bsum = reinterpret_cast<double*>(ebar + R);
  volatile int* abort_flag = reinterpret_cast<volatile int*>(bsum + 4);

  const int nxb = (nx + 63) / 64;
  const int ntiles = nxb * ny * L.nzc;
  const long long sites = gr.sites;
  const float dt = L.dt;
  ST* __restrict__ out = static_cast<ST*>(L.out);
  float* __restrict__ eout = L.e_out;
  const int i0 = g * DPT;
  const int oct0 = __float_as_int(t.au[i0].w);
  const bool yneg = oct0 & 2;
  const int zs = (oct0 & 4) ? 1 : 0;
  const int row_own = yneg ? 0 : 1, row_up = yneg ? 1 : 0;
  const int erow_up = yneg ? 2 : 0;
  constexpr int nunits = 2;

  for (int i = g * 32 + lane; i < G * DPT; i += G * 32) {
    const float4 au = t.au[i], nw = t.nw[i];
    const int oct = __float_as_int(au.w);
    const float azw = (oct & 4) ? 1.f - au.z : au.z;
    DirConstM16 d;
    d.s0 = make_float4(au.x, au.x, au.y, au.y);
    d.s1 = make_float4(azw, azw, nw.x, nw.x);
    d.s2 = make_float4(nw.y, nw.y, nw.z, nw.z);
    d.s3 = make_float4(nw.w, nw.w, dt, dt);
    d.sh = (oct & 1) ? 1 : -1;
    d.inert = oct & 8;
    d.pad0 = d.pad1 = 0;
    dirs[i] = d;
  }
  if (lane == 0) {
    for (int r = 0; r < R; ++r) mbar_init(smem_u32(&mbar[g * R + r]), 1);
    if (g == 0)
      for (int r = 0; r < R; ++r) mbar_init(smem_u32(&ebar[r]), 1);
  }
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

  unsigned char* my_ring = ring + (size_t)g * R * SLOTB;
  bool alive = true;
  int issued = 0, waited = 0;
  int is_t = blockIdx.x, is_m = 0, is_M = 0, is_x0 = 0, is_yp = 0, is_zp = 0, is_y = 0, is_zb = 0;
  auto issue_seek = [&]() {
    if (is_t < ntiles) {
      const TileGeom tg = tile_geom(is_t, nxb, ny, nz, L.nzc);
      is_M = tile_items<ZC>(tg.zlen);
      is_x0 = tg.x0;
      is_y = tg.y;
      is_yp = yneg ? tg.y + 1 : tg.y;
      is_zb = tg.zbeg;
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
      mbar_arrive_tx(bar, BOXH * DPT * 2 * ZC * 2);
      tma_load_4d(smem_u32(my_ring + (size_t)slot * SLOTB), &tmap, is_x0, i0, is_yp,
                  is_zp + is_m * ZC, bar);
      if (g == 0) {
        const uint32_t eb = smem_u32(&ebar[slot]);
        mbar_arrive_tx(eb, BOXH * 3 * (ZC + 1) * 4);
        tma_load_3d(smem_u32(ering + (size_t)slot * ESLOT), &emap, is_x0, is_y,
                    is_zb + is_m * ZC, eb);
      }
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
    const uint32_t par = (uint32_t)((q / R) & 1);
    if (!mbar_wait(smem_u32(&mbar[g * R + q % R]), par, L.err) ||
        !mbar_wait(smem_u32(&ebar[q % R]), par, L.err)) {
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
    ST* const orow = out + (long long)i0 * gr.si + (long long)(y + 1) * gr.sy + xa + GL;
    for (int m = 0; m < M; ++m, ++q) {
      const int z = zbeg - 1 + m;
      const bool zok = z >= zbeg && z < zend;
      if (g == G - 1) {
        int tn = ti, mn = m + 1;
        if (mn == M) {
          tn = ti + gridDim.x;
          mn = 0;
        }
        if (tn < ntiles) stage(tn, mn, (q + 1) & 1);
      }
      const float* fb = fbuf + (q & 1) * 6 * 64;
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
      // beta_i, A_i and g'_i = A_i dt (W beta_i)^-3 for direction constants d
      auto coll = [&](const DirConstM16& d, float2& beta, float2& A, float2& gp) {
        const float4 s1 = d.s1, s2 = d.s2, s3 = d.s3;
        const float2 vn = f2fma(vz, make_float2(s2.z, s2.w),
                                f2fma(vy, make_float2(s2.x, s2.y), f2mul(vx, make_float2(s1.z, s1.w))));
        beta = f2sub(one2, vn);
        const float2 den = f2fma(cA, beta, one2);
        A = make_float2(__fdividef(1.f, den.x), __fdividef(1.f, den.y));
        const float2 wb = f2mul(W, beta);
        const float2 iw = make_float2(__fdividef(1.f, wb.x), __fdividef(1.f, wb.y));
        gp = f2mul(f2mul(A, make_float2(s3.z, s3.w)), f2mul(iw, f2mul(iw, iw)));
      };
      while (issued < q + R && issue()) {
      }
      wait_item(q);
      unsigned char* slot = my_ring + (size_t)(q % R) * SLOTB;
      const ST* sl = reinterpret_cast<const ST*>(slot);
      const float* es = ering + (size_t)(q % R) * ESLOT;
      const float* eo = es + (zs * 3 + 1) * BOXH + wc;
      const float* eu = es + (zs * 3 + erow_up) * BOXH + wc;
      const float2 EPo = *reinterpret_cast<const float2*>(eo);
      const float2 EPu = *reinterpret_cast<const float2*>(eu);
      const float Emo = eo[-1], Epo = eo[2], Emu = eu[-1], Epu = eu[2];
      float2 Is[DPT];  // f*_i
      float2 aS = make_float2(0.f, 0.f), aX = aS, aY = aS, aA = aS, aG = aS;
#pragma unroll
      for (int k = 0; k < DPT; ++k) {
        const DirConstM16& d = dirs[i0 + k];
        const float4 s0 = d.s0, s1 = d.s1, s3 = d.s3;
        const float2 ax = make_float2(s0.x, s0.y), ay = make_float2(s0.z, s0.w);
        const float2 az = make_float2(s1.x, s1.y), w2 = make_float2(s3.x, s3.y);
        const ST* po = sl + (row_own * DPT + k) * BOXH + wc;
        const ST* pu = sl + (row_up * DPT + k) * BOXH + wc;
        const float2 qo = C2::to2(*reinterpret_cast<const T2*>(po));
        const float2 qu = C2::to2(*reinterpret_cast<const T2*>(pu));
        const float2 fo = f2fma(EPo, qo, EPo);
        const float2 fu = f2fma(EPu, qu, EPu);
        float2 So, Su;
        if (d.sh > 0) {
          So = make_float2(fo.y, fmaf(Epo, C2::to1(po[2]), Epo));
          Su = make_float2(fu.y, fmaf(Epu, C2::to1(pu[2]), Epu));
        } else {
          So = make_float2(fmaf(Emo, C2::to1(po[-1]), Emo), fo.x);
          Su = make_float2(fmaf(Emu, C2::to1(pu[-1]), Emu), fu.x);
        }
        const float2 X0 = f2fma(ax, f2sub(So, fo), fo);
        const float2 X1 = f2fma(ax, f2sub(Su, fu), fu);
        const float2 Bn = f2fma(ay, f2sub(X1, X0), X0);
        const float2 r = f2fma(az, f2sub(carry[k], Bn), Bn);
        carry[k] = Bn;
        Is[k] = r;
        float2 beta, A, gp;
        coll(d, beta, A, gp);
        const float2 af = f2mul(A, r);
        const float2 wb2 = f2mul(w2, f2mul(beta, beta));
        aS = f2fma(w2, r, aS);
        aX = f2fma(wb2, f2fma(gp, et, af), aX);
        aY = f2fma(wb2, gp, aY);
        aA = f2fma(w2, af, aA);
        aG = f2fma(w2, gp, aG);
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
          const float* p = reinterpret_cast<const float*>(ring + ((size_t)qq * R + s) * SLOTB) + f;
          S += p[0];
          X += p[64];
          Y += p[128];
          SA += p[192];
          SG += p[256];
        }
        const float W2 = __fdividef(1.f, 1.f - fmaf(uz, uz, fmaf(uy, uy, ux * ux)));
        const float J = __fdividef(W2 * X, 1.f - kt0 * W2 * Y);
        const float src = fmaf(kt0, J, etat);
        const float Enew = fmaf(SG, src, SA);
        const float Eh = fmaxf(Enew, EPS_E);
        coef[f] = src;
        coef[64 + f] = __fdividef(1.f, Eh);
        if (v) {
          bud_a += S;
          bud_b += Enew;
          if (alive) store_e(eout, gr, z, y, x, Eh);
        }
      }
      __syncthreads();
      if (L.budget_partials && g < nunits) {
        bud_da += (double)bud_a;
        bud_db += (double)bud_b;
        bud_a = bud_b = 0.f;
      }
      const float2 src = reinterpret_cast<const float2*>(coef)[lane];
      const float2 rinv = reinterpret_cast<const float2*>(coef + 64)[lane];
      const bool zface = gr.periodic[2] && (z == 0 || z == nz - 1);
      const bool fast = __all_sync(0xffffffffu, in0 && in1) && zok &&
                        !(y_face && ny == 1) && !(zface && nz == 1);
      const bool xghost = __any_sync(0xffffffffu, gx_lo || gx_hi);
      const int yface_rows = (y == ny - 1 ? 0 : ny + 1) - (y + 1);
      if (alive && fast) {
        ST* base = orow + (long long)(z + 1) * gr.sz;
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
          if (inert_mask >> k & 1u) continue;
          float2 beta, A, gp;
          coll(dirs[i0 + k], beta, A, gp);
          const float2 qn = f2fma(f2fma(gp, src, f2mul(A, Is[k])), rinv, make_float2(-1.f, -1.f));
          const T2 hq = C2::from2(qn);
          ST* dst = base + (long long)k * gr.si;
          if constexpr (!PER) {
            *reinterpret_cast<T2*>(dst) = hq;
          } else {
            auto put = [&](ST* dd) {
              *reinterpret_cast<T2*>(dd) = hq;
              if (xghost && gx_any) dd[gx_off] = gx_y ? hq.y : hq.x;  // one predicated store
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
#pragma unroll
        for (int k = 0; k < DPT; ++k) {
          if (inert_mask >> k & 1u) continue;
          float2 beta, A, gp;
          coll(dirs[i0 + k], beta, A, gp);
          const float2 qn = f2fma(f2fma(gp, src, f2mul(A, Is[k])), rinv, make_float2(-1.f, -1.f));
          const T2 hq = C2::from2(qn);
          store_pop(out, gr, i0 + k, z, y, xa, hq.x);
          if (in1) store_pop(out, gr, i0 + k, z, y, xa + 1, hq.y);
        }
      }
    }
  }
  for (int qq = waited; qq < issued; ++qq) {
    const uint32_t par = (uint32_t)((qq / R) & 1);
    mbar_wait(smem_u32(&mbar[g * R + qq % R]), par, L.err);
    if (g == 0) mbar_wait(smem_u32(&ebar[qq % R]), par, L.err);
  }
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
size_t smem_moving16(int G) {
  return (size_t)G * R * slot_bytes16<DPT, 1>() +
         sizeof(float) * ((size_t)R * eslot_floats<1>() + 2 * 64 + 2 * 6 * 64) +
         sizeof(DirConstM16) * (size_t)G * DPT + 8 * ((size_t)G * R + R) + sizeof(double) * 4 + 16;
}

template <class ST, bool PER, int DPT, int R, int MAXT, int REGS>
cudaError_t set_attr_moving16() {
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && (attr_set >> dev & 1ull)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(k_step_moving16<ST, PER, DPT, R, MAXT, REGS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024 - 1024);
  if (e == cudaSuccess && dev < 64) attr_set |= 1ull << dev;
  return e;
}

template <class ST, int DPT, int R, int MAXT, int REGS>
cudaError_t occupancy_moving16_t(int G, int* per_sm) {
  int a = 0, b = 0;
  cudaError_t e = set_attr_moving16<ST, false, DPT, R, MAXT, REGS>();
  if (e == cudaSuccess) e = set_attr_moving16<ST, true, DPT, R, MAXT, REGS>();
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &a, k_step_moving16<ST, false, DPT, R, MAXT, REGS>, 32 * G, smem_moving16<DPT, R>(G));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &b, k_step_moving16<ST, true, DPT, R, MAXT, REGS>, 32 * G, smem_moving16<DPT, R>(G));
  *per_sm = std::min(a, b);
  return e;
}

template <class ST, int DPT, int R, int MAXT, int REGS>
cudaError_t launch_moving16_t(const StepLaunch& L, const MovingCoef& c, const DirTable& t,
                              cudaStream_t s, int* nblocks) {
  const int G = L.N / DPT;
  if (!L.tmap_in || !L.tmap_e || !L.e_out || G < 1 || G * DPT != L.N || 32 * G > MAXT ||
      L.nzc < 1 || L.nzc > L.g.nz || L.ctas < 1)
    return cudaErrorInvalidValue;
  if (L.budget_partials && L.ctas > L.partials_cap) return cudaErrorInvalidValue;
  if (nblocks) *nblocks = L.ctas;
  const size_t smem = smem_moving16<DPT, R>(G);
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  const bool per = L.g.periodic[0] || L.g.periodic[1] || L.g.periodic[2];
  const cudaError_t e = per ? set_attr_moving16<ST, true, DPT, R, MAXT, REGS>()
                            : set_attr_moving16<ST, false, DPT, R, MAXT, REGS>();
  if (e != cudaSuccess) return e;
  if (per)
    k_step_moving16<ST, true, DPT, R, MAXT, REGS>
        <<<L.ctas, dim3(32, G), smem, s>>>(*L.tmap_in, *L.tmap_e, L, c, t);
  else
    k_step_moving16<ST, false, DPT, R, MAXT, REGS>
        <<<L.ctas, dim3(32, G), smem, s>>>(*L.tmap_in, *L.tmap_e, L, c, t);
  return cudaGetLastError();
}

#define LBRT_MOVING16_PLANS(X) \
  X(5, 320, 96)                \
  X(11, 512, 128)              \
  X(10, 544, 96)

template <int DPT, int ZC, int R>
size_t step_smem16(int G) {
  return (size_t)G * R * slot_bytes16<DPT, ZC>() + sizeof(float) * ((size_t)R * eslot_floats<ZC>() + ZC * 5 * 64) +
         sizeof(DirConst16) * (size_t)G * DPT + 8 * ((size_t)G * R + R) + sizeof(double) * 4 * ZC + 16;
}

template <class ST, bool BATCH, bool PER, int DPT, int ZC, int R, int MAXT, int REGS>
cudaError_t set_smem_attr16() {
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && (attr_set >> dev & 1ull)) return cudaSuccess;
  const cudaError_t e = cudaFuncSetAttribute(k_step_16<ST, BATCH, PER, DPT, ZC, R, MAXT, REGS>,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             227 * 1024 - 1024);
  if (e == cudaSuccess && dev < 64) attr_set |= 1ull << dev;
  return e;
}

template <class ST, bool BATCH, int DPT, int ZC, int R, int MAXT, int REGS>
cudaError_t occupancy16(int G, int* per_sm) {
  int a = 0, b = 0;
  cudaError_t e = set_smem_attr16<ST, BATCH, false, DPT, ZC, R, MAXT, REGS>();
  if (e == cudaSuccess) e = set_smem_attr16<ST, BATCH, true, DPT, ZC, R, MAXT, REGS>();
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &a, k_step_16<ST, BATCH, false, DPT, ZC, R, MAXT, REGS>, 32 * G,
        step_smem16<DPT, ZC, R>(G));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &b, k_step_16<ST, BATCH, true, DPT, ZC, R, MAXT, REGS>, 32 * G,
        step_smem16<DPT, ZC, R>(G));
  *per_sm = std::min(a, b);
  return e;
}

template <class ST, int DPT, int ZC, int R, int MAXT, int REGS>
cudaError_t launch16(const StepLaunch& L, const StaticCoef& c, const DirTable& t, cudaStream_t s,
                     int* nblocks) {
  const int G = L.N / DPT;
  if (!L.tmap_in || !L.tmap_e || !L.e_out || G < 1 || G * DPT != L.N || 32 * G > MAXT ||
      L.nzc < 1 || L.nzc > L.g.nz || L.ctas < 1)
    return cudaErrorInvalidValue;
  if (L.budget_partials && L.ctas > L.partials_cap) return cudaErrorInvalidValue;
  if (nblocks) *nblocks = L.ctas;
  const size_t smem = step_smem16<DPT, ZC, R>(G);
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  const bool per = L.g.periodic[0] || L.g.periodic[1] || L.g.periodic[2];
  const cudaError_t e = per ? set_smem_attr16<ST, false, true, DPT, ZC, R, MAXT, REGS>()
                            : set_smem_attr16<ST, false, false, DPT, ZC, R, MAXT, REGS>();
  if (e != cudaSuccess) return e;
  ProblemDesc one{};
  one.g = L.g;
  one.out = L.out;
  one.e_out = L.e_out;
  one.cf = c;
  one.dt = L.dt;
  one.collision = L.collision;
  one.lambda_iters = L.lambda_iters;
  one.nzc = L.nzc;
  one.tile_start = 0;
  one.ntiles = (L.g.nx + 63) / 64 * L.g.ny * L.nzc;
  one.budget_partials = L.budget_partials;
  if (per)
    k_step_16<ST, false, true, DPT, ZC, R, MAXT, REGS><<<L.ctas, dim3(32, G), smem, s>>>(
        *L.tmap_in, *L.tmap_e, one, nullptr, 1, one.ntiles, L.err, t);
  else
    k_step_16<ST, false, false, DPT, ZC, R, MAXT, REGS><<<L.ctas, dim3(32, G), smem, s>>>(
        *L.tmap_in, *L.tmap_e, one, nullptr, 1, one.ntiles, L.err, t);
  return cudaGetLastError();
}

template <class ST, int DPT, int ZC, int R, int MAXT, int REGS>
cudaError_t launch16_batch(const BatchLaunch& B, const DirTable& t, cudaStream_t s) {
  const int G = B.N / DPT;
  if (G < 1 || G * DPT != B.N || 32 * G > MAXT || B.ctas < 1 || B.ntiles < 1 || !B.table ||
      B.nprob < 1)
    return cudaErrorInvalidValue;
  const size_t smem = step_smem16<DPT, ZC, R>(G);
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  const cudaError_t e = B.periodic ? set_smem_attr16<ST, true, true, DPT, ZC, R, MAXT, REGS>()
                                   : set_smem_attr16<ST, true, false, DPT, ZC, R, MAXT, REGS>();
  if (e != cudaSuccess) return e;
  CUtensorMap unused{};
  ProblemDesc none{};
  if (B.periodic)
    k_step_16<ST, true, true, DPT, ZC, R, MAXT, REGS><<<B.ctas, dim3(32, G), smem, s>>>(
        unused, unused, none, B.table, B.nprob, B.ntiles, B.err, t);
  else
    k_step_16<ST, true, false, DPT, ZC, R, MAXT, REGS><<<B.ctas, dim3(32, G), smem, s>>>(
        unused, unused, none, B.table, B.nprob, B.ntiles, B.err, t);
  return cudaGetLastError();
}

constexpr int kRing16 = 2;

template <class ST, bool PER, int DA, int ZA, int DB, int ZB, int R, int MAXT, int REGS>
cudaError_t set_smem_attr16_pair() {
  static unsigned long long attr_set = 0;
  int dev = 0;
  cudaGetDevice(&dev);
  if (dev < 64 && (attr_set >> dev & 1ull)) return cudaSuccess;
  const cudaError_t e =
      cudaFuncSetAttribute(k_step_16_pair<ST, PER, DA, ZA, DB, ZB, R, MAXT, REGS>,
                           cudaFuncAttributeMaxDynamicSharedMemorySize, 227 * 1024 - 1024);
  if (e == cudaSuccess && dev < 64) attr_set |= 1ull << dev;
  return e;
}

template <int DA, int ZA, int DB, int ZB, int R>
size_t pair_smem16(int ga, int gb) {
  return std::max(step_smem16<DA, ZA, R>(ga), step_smem16<DB, ZB, R>(gb));
}

template <class ST, int DA, int ZA, int DB, int ZB, int R, int MAXT, int REGS>
cudaError_t occupancy16_pair(int ga, int gb, int* per_sm) {
  int a = 0, b = 0;
  const int threads = 32 * std::max(ga, gb);
  cudaError_t e = set_smem_attr16_pair<ST, false, DA, ZA, DB, ZB, R, MAXT, REGS>();
  if (e == cudaSuccess) e = set_smem_attr16_pair<ST, true, DA, ZA, DB, ZB, R, MAXT, REGS>();
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &a, k_step_16_pair<ST, false, DA, ZA, DB, ZB, R, MAXT, REGS>, threads,
        pair_smem16<DA, ZA, DB, ZB, R>(ga, gb));
  if (e == cudaSuccess)
    e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(
        &b, k_step_16_pair<ST, true, DA, ZA, DB, ZB, R, MAXT, REGS>, threads,
        pair_smem16<DA, ZA, DB, ZB, R>(ga, gb));
  *per_sm = std::min(a, b);
  return e;
}

// A = the group of plan (DA, ZA), B = the group of plan (DB, ZB); CTAs
// 0 .. ctas_a - 1 of the B.ctas-CTA grid take A's tiles.
template <class ST, int DA, int ZA, int DB, int ZB, int R, int MAXT, int REGS>
cudaError_t launch16_pair(const BatchLaunch& A, const DirTable& ta, const BatchLaunch& B,
                          const DirTable& tb, int ctas_a, int ctas, cudaStream_t s) {
  const int ga = A.N / DA, gb = B.N / DB;
  if (ga < 1 || ga * DA != A.N || gb < 1 || gb * DB != B.N || 32 * std::max(ga, gb) > MAXT ||
      ctas_a < 1 || ctas_a >= ctas || !A.table || !B.table || A.nprob < 1 || B.nprob < 1 ||
      A.ntiles < 1 || B.ntiles < 1)
    return cudaErrorInvalidValue;
  const size_t smem = pair_smem16<DA, ZA, DB, ZB, R>(ga, gb);
  if (smem > 226 * 1024) return cudaErrorInvalidValue;
  const bool per = A.periodic || B.periodic;
  const cudaError_t e = per ? set_smem_attr16_pair<ST, true, DA, ZA, DB, ZB, R, MAXT, REGS>()
                            : set_smem_attr16_pair<ST, false, DA, ZA, DB, ZB, R, MAXT, REGS>();
  if (e != cudaSuccess) return e;
  CUtensorMap unused{};
  ProblemDesc none{};
  const dim3 block(32, std::max(ga, gb));
  if (per)
    k_step_16_pair<ST, true, DA, ZA, DB, ZB, R, MAXT, REGS><<<ctas, block, smem, s>>>(
        unused, none, A.table, A.nprob, A.ntiles, ga, ctas_a, B.table, B.nprob, B.ntiles, gb,
        B.err, ta, tb);
  else
    k_step_16_pair<ST, false, DA, ZA, DB, ZB, R, MAXT, REGS><<<ctas, block, smem, s>>>(
        unused, none, A.table, A.nprob, A.ntiles, ga, ctas_a, B.table, B.nprob, B.ntiles, gb,
        B.err, ta, tb);
  return cudaGetLastError();
}


// Tile plans for 16-bit storage (directions per warp, planes per batch,
// thread cap, registers per thread), in order of preference.  The decoded
// energy densities of a batch take registers that the float32 kernel does
// not need, so the 42-direction plan works one plane per batch.
#define LBRT_TILE_PLANS16(X) \
  X(5, 1, 320, 96)           \
  X(11, 1, 512, 128)         \
  X(10, 1, 544, 96)          \
  X(8, 1, 512, 128)          \
  X(4, 1, 640, 96)

template <class ST>
cudaError_t launch_typed(const StepLaunch& L, const StaticCoef& c, const DirTable& t, int dpt, int zc,
                         cudaStream_t s, int* nblocks) {
#define LBRT_L16(D, Z, T, B) \
  if (dpt == D && zc == Z) return launch16<ST, D, Z, kRing16, T, B>(L, c, t, s, nblocks);
  LBRT_TILE_PLANS16(LBRT_L16)
#undef LBRT_L16
  return cudaErrorInvalidValue;
}

// Alternative batched kernels (directions per warp, planes per batch, thread
// cap, registers) with the memory layout of the tile plan of the same
// directions per warp, timed by the batch autotuner against the plan's own
// kernel: two planes per batch for the 42-direction plan, whose 128
// registers hold one 9-warp CTA per SM instead of two.
#define LBRT_BATCH_ALT16(X) X(5, 2, 320, 128)

template <class ST>
cudaError_t occupancy_typed(int dpt, int zc, int G, int* per_sm, bool batch, int alt) {
  if (alt) {
#define LBRT_OA16(D, Z, T, B) \
  if (dpt == D && zc == Z) return occupancy16<ST, true, D, Z, kRing16, T, B>(G, per_sm);
    LBRT_BATCH_ALT16(LBRT_OA16)
#undef LBRT_OA16
    return cudaErrorInvalidValue;
  }
#define LBRT_O16(D, Z, T, B) \
  if (dpt == D && zc == Z)                                                              \
    return batch ? occupancy16<ST, true, D, Z, kRing16, T, B>(G, per_sm)                \
                 : occupancy16<ST, false, D, Z, kRing16, T, B>(G, per_sm);
  LBRT_TILE_PLANS16(LBRT_O16)
#undef LBRT_O16
  return cudaErrorInvalidValue;
}

// Plan pairs that share one batched launch (plan A, plan B, thread cap,
// registers): the 42-direction (5 per warp) and the 162-direction (11 per
// warp) icosahedral sets.
#define LBRT_PAIR_PLANS16(X) X(5, 1, 11, 1, 512, 128)

template <class ST>
cudaError_t launch_typed_pair(const BatchLaunch& A, const DirTable& ta, const BatchLaunch& B,
                              const DirTable& tb, int ctas_a, int ctas, cudaStream_t s) {
#define LBRT_LP16(DA, ZA, DB, ZB, T, R_)                                                  \
  if (A.dpt == DA && A.zc == ZA && B.dpt == DB && B.zc == ZB)                            \
    return launch16_pair<ST, DA, ZA, DB, ZB, kRing16, T, R_>(A, ta, B, tb, ctas_a, ctas, s);
  LBRT_PAIR_PLANS16(LBRT_LP16)
#undef LBRT_LP16
  return cudaErrorInvalidValue;
}

template <class ST>
cudaError_t occupancy_typed_pair(int da, int za, int ga, int db, int zb, int gb, int* per_sm) {
#define LBRT_OP16(DA, ZA, DB, ZB, T, R_)                                                  \
  if (da == DA && za == ZA && db == DB && zb == ZB)                                      \
    return occupancy16_pair<ST, DA, ZA, DB, ZB, kRing16, T, R_>(ga, gb, per_sm);
  LBRT_PAIR_PLANS16(LBRT_OP16)
#undef LBRT_OP16
  return cudaErrorInvalidValue;
}

template <class ST>
cudaError_t launch_typed_batch(const BatchLaunch& B, const DirTable& t, cudaStream_t s) {
  if (B.alt) {
#define LBRT_LA16(D, Z, T, R_) \
  if (B.dpt == D && B.zc == Z) return launch16_batch<ST, D, Z, kRing16, T, R_>(B, t, s);
    LBRT_BATCH_ALT16(LBRT_LA16)
#undef LBRT_LA16
    return cudaErrorInvalidValue;
  }
#define LBRT_LB16(D, Z, T, R_) \
  if (B.dpt == D && B.zc == Z) return launch16_batch<ST, D, Z, kRing16, T, R_>(B, t, s);
  LBRT_TILE_PLANS16(LBRT_LB16)
#undef LBRT_LB16
  return cudaErrorInvalidValue;
}

}  // namespace

#define LBRT_PLAN_ROW16(D, Z, T, B) {D, Z, T},
const int kTilePlans16[][3] = {LBRT_TILE_PLANS16(LBRT_PLAN_ROW16)};
#undef LBRT_PLAN_ROW16
const int kNumTilePlans16 = sizeof(kTilePlans16) / sizeof(kTilePlans16[0]);

size_t step_tile_smem16(int dpt, int zc, int warps) {
#define LBRT_S16(D, Z, T, B) \
  if (dpt == D && zc == Z) return step_smem16<D, Z, kRing16>(warps);
  LBRT_TILE_PLANS16(LBRT_S16)
#undef LBRT_S16
  return (size_t)-1;
}

cudaError_t launch_tma16_static(const StepLaunch& L, const StaticCoef& c, const DirTable& t,
                                int storage, cudaStream_t s, int* nblocks) {
  if (storage == ST_F16) return launch_typed<__half>(L, c, t, L.dpt, L.zc, s, nblocks);
  if (storage == ST_BF16) return launch_typed<__nv_bfloat16>(L, c, t, L.dpt, L.zc, s, nblocks);
  return cudaErrorInvalidValue;
}

int batch_alt_zc16(int dpt) {
#define LBRT_AZ16(D, Z, T, R_) \
  if (dpt == D) return Z;
  LBRT_BATCH_ALT16(LBRT_AZ16)
#undef LBRT_AZ16
  return 0;
}

cudaError_t occupancy_tma16(int storage, int dpt, int zc, int G, int* per_sm, bool batch, int alt) {
  if (storage == ST_F16) return occupancy_typed<__half>(dpt, zc, G, per_sm, batch, alt);
  if (storage == ST_BF16) return occupancy_typed<__nv_bfloat16>(dpt, zc, G, per_sm, batch, alt);
  return cudaErrorInvalidValue;
}

cudaError_t occupancy_tma16_moving(int storage, int dpt, int G, int* per_sm) {
#define LBRT_M16O(D, T, B)                                                                    \
  if (dpt == D)                                                                             \
    return storage == ST_BF16 ? occupancy_moving16_t<__nv_bfloat16, D, kRing16, T, B>(G, per_sm) \
                              : occupancy_moving16_t<__half, D, kRing16, T, B>(G, per_sm);
  LBRT_MOVING16_PLANS(LBRT_M16O)
#undef LBRT_M16O
  return cudaErrorInvalidValue;
}

cudaError_t launch_tma16_moving(const StepLaunch& L, const MovingCoef& c, const DirTable& t,
                                int storage, cudaStream_t s, int* nblocks) {
#define LBRT_M16L(D, T, B)                                                            \
  if (L.dpt == D && L.zc == 1)                                                        \
    return storage == ST_BF16                                                         \
               ? launch_moving16_t<__nv_bfloat16, D, kRing16, T, B>(L, c, t, s, nblocks) \
               : launch_moving16_t<__half, D, kRing16, T, B>(L, c, t, s, nblocks);
  LBRT_MOVING16_PLANS(LBRT_M16L)
#undef LBRT_M16L
  return cudaErrorInvalidValue;
}

cudaError_t launch_tma16_static_batch(const BatchLaunch& B, const DirTable& t, cudaStream_t s) {
  if (B.storage == ST_F16) return launch_typed_batch<__half>(B, t, s);
  if (B.storage == ST_BF16) return launch_typed_batch<__nv_bfloat16>(B, t, s);
  return cudaErrorInvalidValue;
}

bool tma16_pair_supported(int da, int za, int db, int zb) {
#define LBRT_PS16(DA, ZA, DB, ZB, T, R_) \
  if (da == DA && za == ZA && db == DB && zb == ZB) return true;
  LBRT_PAIR_PLANS16(LBRT_PS16)
#undef LBRT_PS16
  return false;
}

cudaError_t launch_tma16_static_batch_pair(const BatchLaunch& A, const DirTable& ta,
                                           const BatchLaunch& B, const DirTable& tb, int ctas_a,
                                           int ctas, cudaStream_t s) {
  if (A.storage != B.storage) return cudaErrorInvalidValue;
  if (A.storage == ST_F16) return launch_typed_pair<__half>(A, ta, B, tb, ctas_a, ctas, s);
  if (A.storage == ST_BF16) return launch_typed_pair<__nv_bfloat16>(A, ta, B, tb, ctas_a, ctas, s);
  return cudaErrorInvalidValue;
}

cudaError_t occupancy_tma16_pair(int storage, int da, int za, int ga, int db, int zb, int gb,
                                 int* per_sm) {
  if (storage == ST_F16) return occupancy_typed_pair<__half>(da, za, ga, db, zb, gb, per_sm);
  if (storage == ST_BF16)
    return occupancy_typed_pair<__nv_bfloat16>(da, za, ga, db, zb, gb, per_sm);
  return cudaErrorInvalidValue;
}

// TMA descriptors of a padded 16-bit population buffer ([PZ][PY][Ni][PX],
// box 72 x dpt x 2 x zc) and of a padded float32 E buffer ([PZ][PY][PX],
// box 72 x 3 x (zc + 1)).
bool make_pop16_tensor_map(CUtensorMap* map, const Grid& g, int Ni, void* base, int storage, int dpt,
                           int zc, std::string& err) {
  auto encode = tensor_map_encoder(err);
  if (!encode) return false;
  const cuuint64_t dims[4] = {(cuuint64_t)g.PX, (cuuint64_t)Ni, (cuuint64_t)g.PY, (cuuint64_t)g.PZ};
  const cuuint64_t strides[3] = {(cuuint64_t)g.si * 2, (cuuint64_t)g.sy * 2, (cuuint64_t)g.sz * 2};
  const cuuint32_t box[4] = {(cuuint32_t)BOXH, (cuuint32_t)dpt, 2, (cuuint32_t)zc};
  const cuuint32_t estr[4] = {1, 1, 1, 1};
  const CUresult r = encode(map, storage == ST_BF16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16
                                                    : CU_TENSOR_MAP_DATA_TYPE_FLOAT16,
                            4, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                            CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                            CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled (16-bit populations) failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

bool make_e_tensor_map(CUtensorMap* map, const Grid& g, float* base, int zc, std::string& err) {
  auto encode = tensor_map_encoder(err);
  if (!encode) return false;
  const cuuint64_t dims[3] = {(cuuint64_t)g.PX, (cuuint64_t)g.PY, (cuuint64_t)g.PZ};
  const cuuint64_t strides[2] = {(cuuint64_t)g.PX * 4, (cuuint64_t)g.PX * g.PY * 4};
  const cuuint32_t box[3] = {(cuuint32_t)BOXH, 3, (cuuint32_t)(zc + 1)};
  const cuuint32_t estr[3] = {1, 1, 1};
  const CUresult r = encode(map, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 3, base, dims, strides, box, estr,
                            CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
                            CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
  if (r != CUDA_SUCCESS) {
    err = "cuTensorMapEncodeTiled (E) failed (" + std::to_string((int)r) + ")";
    return false;
  }
  return true;
}

}  // namespace lbrt
