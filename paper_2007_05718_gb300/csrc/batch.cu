// Batch runtime of the C ABI (lb_rt_batch_* in include/lb_rt.h): many
// independent static-fluid problems resident on one device, admitted by
// device memory, grouped by direction table and advanced together with one
// persistent kernel launch per group and step (the batched form of the
// TMA-fed step kernels) or one launch per step for two groups of different
// direction counts, a CUDA graph per launch plan and an autotuner of the
// tile shape (z chunks, planes per batch of the batched kernel) and of the
// pairing.  The paper solves one problem at a time; this layer is the
// library's own.
#include <algorithm>
#include <cstring>
#include <new>

#include "handle.h"
#include "lb_rt_internal.h"

using namespace lbrt;

namespace {

struct Member {
  lb_rt* h = nullptr;
  long long nsteps = 0;
  size_t bytes = 0;
  int group = -1;
  bool used = false;
  cudaEvent_t ready = nullptr;  // admission work (on the problem's own stream) done
  bool joined = false;          // the batch stream has waited for `ready`
  long long done_tick = -1;     // tick that enqueued the problem's last step
};

// Problems that share the internal direction table, tile plan and storage.
struct Group {
  DirTable table{};
  int Ni = 0, dpt = 0, zc = 0;
  int per_sm = 0;         // resident CTAs per SM of the batched kernel
  int zchunk = 16;        // planes per tile
  // autotuner: candidates are timed on successive ticks of a new member set
  std::vector<int> cands;
  std::vector<double> cost;  // ms per (site x step) of each candidate
  int cand = 0;
  bool tuned = false;
  long long tuned_sites = 0;
  cudaEvent_t ev0 = nullptr, ev1 = nullptr;
  int ctas = 0;           // CTAs of the last launch
  bool paired = false;    // the last tick ran the group in a launch shared with another group
  // alternative batched kernel of the same layout (batch_alt_zc): its planes
  // per batch (0: none) and residency; alt = 1 while it is in use.  The
  // autotuner times it at the best z chunk after the z-chunk candidates.
  int alt_zc = 0, alt_per_sm = 0, alt = 0;
  int stage = 0;          // tuning: 0 z chunks, 1 the alternative kernel
  int zc_now() const { return alt ? alt_zc : zc; }
  int last_zc = 0;        // planes per batch of the kernel of the last launch
};

constexpr int kZCandidates[] = {8, 16, 32, 64};

}  // namespace

struct lb_rt_batch {
  lb_rt_batch_config cfg{};
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  size_t budget = 0, used = 0;
  int sms = 0;
  std::vector<Member> slots;
  std::vector<Group> groups;
  // descriptor tables, one pair per tick parity (host staging, pinned, and
  // device copy): tick t fills pair t & 1 once tick t - 2 has completed, so
  // the host prepares a tick while the previous one runs
  ProblemDesc* h_desc[2] = {nullptr, nullptr};
  ProblemDesc* d_desc[2] = {nullptr, nullptr};
  size_t desc_cap[2] = {0, 0};
  static constexpr int kTickEvents = 4;
  cudaEvent_t tick_ev[kTickEvents] = {nullptr, nullptr, nullptr, nullptr};  // end of tick t: [t % 4]
  long long ticks = 0;   // ticks enqueued
  // released problems whose device memory is returned at the next
  // synchronisation (freeing right away would wait for the ticks in flight)
  std::vector<lb_rt*> grave;
  size_t grave_bytes = 0;
  // tensor maps of every slot: [slot][kernel variant][parity][pop, E]
  CUtensorMap* h_maps = nullptr;
  CUtensorMap* d_maps = nullptr;
  bool maps_dirty = true;
  unsigned* d_err = nullptr;
  // one graph per tick parity; the launch plan it was captured for: per
  // launch (group, first descriptor, problems, tiles) and per descriptor
  // (slot, z chunks); a graph is replayed only for an identical plan, and a
  // changed plan updates the instantiated graph in place where the update
  // applies
  cudaGraph_t graph[2] = {nullptr, nullptr};
  cudaGraphExec_t exec[2] = {nullptr, nullptr};
  std::vector<long long> graph_sig[2];
  // two groups in one launch (cfg.pair_groups): the groups of the pair, the
  // resident CTAs per SM of the paired kernel, and the autotuner's choice
  // (mode 2): -1 undecided, 0 separate launches, 1 paired launch, timed on
  // one tick each and normalised per site-direction update
  int pair_a = -1, pair_b = -1, pair_per_sm = 0;
  int pair_choice = -1, pair_trial = 0;
  long long pair_sites = 0;  // sites of the two groups when the choice was timed
  double pair_cost[2] = {0.0, 0.0};
  cudaEvent_t pev0 = nullptr, pev1 = nullptr;
  std::string msg;
};

namespace {

lb_rt_status bfail(lb_rt_batch* b, lb_rt_status st, const std::string& m) {
  if (b) b->msg = m;
  return st;
}

lb_rt_status bcuda(lb_rt_batch* b, cudaError_t e, const char* where) {
  return bfail(b, e == cudaErrorMemoryAllocation ? LB_RT_ENOMEM : LB_RT_ECUDA,
               std::string(where) + ": " + cudaGetErrorString(e));
}

#define BCK(b, call)                                   \
  do {                                                 \
    cudaError_t e_ = (call);                           \
    if (e_ != cudaSuccess) return bcuda(b, e_, #call); \
  } while (0)

// true when tick t has completed on the device (ticks up to t_last - 2 have:
// tick t_last waited for them before it was enqueued)
bool tick_done(lb_rt_batch* b, long long t) {
  if (t < 0 || t <= b->ticks - 3) return true;
  const cudaError_t e = cudaEventQuery(b->tick_ev[t % lb_rt_batch::kTickEvents]);
  if (e == cudaErrorNotReady) {
    (void)cudaGetLastError();
    return false;
  }
  return true;
}

// free the released problems (the caller has synchronised the batch stream)
void flush_grave(lb_rt_batch* b) {
  for (lb_rt* h : b->grave) lb_rt_destroy(h);
  b->grave.clear();
  b->used -= b->grave_bytes;
  b->grave_bytes = 0;
}

bool same_table(const Group& g, const lb_rt* h) {
  return g.Ni == h->Ni && g.dpt == h->dpt && g.zc == h->zc &&
         std::memcmp(&g.table, &h->table, sizeof(DirTable)) == 0;
}

// One launch of a tick: a group's problems of one step, and optionally a
// second group's (b_*) in the same launch, its problems on CTAs ctas_a ..
// ctas - 1.
struct Launch {
  int group, first, nprob, ntiles, periodic;
  long long sd = 0;  // site-direction updates of the launch's problems of `group`
  int b_group = -1, b_first = 0, b_nprob = 0, b_ntiles = 0, b_periodic = 0;
  long long b_sd = 0;
  int ctas_a = 0, ctas = 0;
};

}  // namespace

extern "C" {

lb_rt_status lb_rt_batch_create(const lb_rt_batch_config* cfg, lb_rt_batch** out) {
  if (!cfg || !out) return LB_RT_EINVAL;
  *out = nullptr;
  if (cfg->max_problems < 1 || cfg->max_problems > LB_RT_BATCH_MAX || cfg->steps_per_tick < 1 ||
      cfg->pair_groups < 0 || cfg->pair_groups > 2 ||
      (cfg->storage != LB_RT_F32 && cfg->storage != LB_RT_F16_DEV &&
       cfg->storage != LB_RT_BF16_DEV))
    return LB_RT_EINVAL;
  lb_rt_batch* b = new (std::nothrow) lb_rt_batch();
  if (!b) return LB_RT_ENOMEM;
  b->cfg = *cfg;
  b->slots.resize(cfg->max_problems);
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&b->sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) {
    if (cfg->stream) {
      b->stream = (cudaStream_t)cfg->stream;
    } else {
      e = cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking);
      b->own_stream = e == cudaSuccess;
    }
  }
  if (e == cudaSuccess) {
    size_t fr = 0, tot = 0;
    e = cudaMemGetInfo(&fr, &tot);
    b->budget = cfg->mem_budget ? cfg->mem_budget : (size_t)(0.8 * (double)fr);
  }
  const size_t nmaps = (size_t)cfg->max_problems * 8;
  if (e == cudaSuccess) e = cudaMallocHost((void**)&b->h_maps, sizeof(CUtensorMap) * nmaps);
  if (e == cudaSuccess) std::memset(b->h_maps, 0, sizeof(CUtensorMap) * nmaps);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_maps, sizeof(CUtensorMap) * nmaps);
  if (e == cudaSuccess) e = cudaMalloc((void**)&b->d_err, sizeof(unsigned));
  for (int i = 0; i < lb_rt_batch::kTickEvents && e == cudaSuccess; ++i)
    e = cudaEventCreateWithFlags(&b->tick_ev[i], cudaEventDisableTiming);
  if (e == cudaSuccess) e = cudaEventCreate(&b->pev0);
  if (e == cudaSuccess) e = cudaEventCreate(&b->pev1);
  if (e == cudaSuccess) e = cudaMemsetAsync(b->d_err, 0, sizeof(unsigned), b->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->stream);
  if (e != cudaSuccess) {
    lb_rt_batch_destroy(b);
    return e == cudaErrorMemoryAllocation ? LB_RT_ENOMEM : LB_RT_ECUDA;
  }
  *out = b;
  return LB_RT_OK;
}

void lb_rt_batch_destroy(lb_rt_batch* b) {
  if (!b) return;
  if (b->stream) cudaStreamSynchronize(b->stream);
  flush_grave(b);
  for (auto& m : b->slots) {
    if (m.h) lb_rt_destroy(m.h);
    if (m.ready) cudaEventDestroy(m.ready);
  }
  for (auto& g : b->groups) {
    if (g.ev0) cudaEventDestroy(g.ev0);
    if (g.ev1) cudaEventDestroy(g.ev1);
  }
  for (int i = 0; i < 2; ++i) {
    if (b->exec[i]) cudaGraphExecDestroy(b->exec[i]);
    if (b->graph[i]) cudaGraphDestroy(b->graph[i]);
    cudaFreeHost(b->h_desc[i]);
    cudaFree(b->d_desc[i]);
  }
  for (cudaEvent_t ev : b->tick_ev)
    if (ev) cudaEventDestroy(ev);
  if (b->pev0) cudaEventDestroy(b->pev0);
  if (b->pev1) cudaEventDestroy(b->pev1);
  cudaFreeHost(b->h_maps);
  cudaFree(b->d_maps);
  cudaFree(b->d_err);
  if (b->own_stream) cudaStreamDestroy(b->stream);
  delete b;
}

size_t lb_rt_batch_problem_bytes(const lb_rt_batch* b, const lb_rt_config* cfg) {
  if (!b || !cfg) return 0;
  lb_rt_config c = *cfg;
  c.storage = b->cfg.storage;
  std::string err;
  return handle_device_bytes(c, err);
}

lb_rt_status lb_rt_batch_admit(lb_rt_batch* b, const lb_rt_config* cfg, const lb_rt_fluid* fluid,
                               int fluid_ptr_kind, const float* state, int state_kind,
                               int state_ptr_kind, long long nsteps, int* slot) {
  if (!b) return LB_RT_EINVAL;
  if (!cfg || !fluid || !state || !slot || nsteps < 0)
    return bfail(b, LB_RT_EINVAL, "null argument or negative step count");
  if (cfg->moving || cfg->budget)
    return bfail(b, LB_RT_EINVAL, "batched problems are static and keep no energy budget");
  lb_rt_config c = *cfg;
  c.storage = b->cfg.storage;
  c.stream = nullptr;  // the problem's own stream: admission overlaps the ticks in flight
  c.budget = 0;
  std::string err;
  const size_t bytes = handle_device_bytes(c, err);
  if (!bytes) return bfail(b, LB_RT_EINVAL, "invalid problem: " + err);
  int s = -1;
  for (int i = 0; i < (int)b->slots.size(); ++i)
    if (!b->slots[i].used) {
      s = i;
      break;
    }
  if (s < 0) return bfail(b, LB_RT_EBUSY, "no free slot");
  if (b->used + bytes > b->budget && !b->grave.empty() && b->used - b->grave_bytes + bytes <= b->budget) {
    // the memory of released problems makes room: return it now
    BCK(b, cudaStreamSynchronize(b->stream));
    flush_grave(b);
  }
  if (b->used + bytes > b->budget)
    return bfail(b, LB_RT_EBUSY, "does not fit the memory budget now");
  lb_rt* h = nullptr;
  lb_rt_status st = lb_rt_create(&c, &h);
  if (st != LB_RT_OK) return bfail(b, st, std::string("create: ") + lb_rt_last_error(nullptr));
  if ((st = lb_rt_set_fluid(h, fluid, fluid_ptr_kind)) != LB_RT_OK ||
      (st = lb_rt_set_state(h, state, state_kind, state_ptr_kind)) != LB_RT_OK) {
    const std::string m = lb_rt_last_error(h);
    lb_rt_destroy(h);
    return bfail(b, st, m);
  }
  int gi = -1;
  for (int i = 0; i < (int)b->groups.size(); ++i)
    if (same_table(b->groups[i], h)) {
      gi = i;
      break;
    }
  if (gi < 0) {
    Group g;
    g.table = h->table;
    g.Ni = h->Ni;
    g.dpt = h->dpt;
    g.zc = h->zc;
    cudaError_t e = occupancy_static_batch(c.storage, g.dpt, g.zc, g.Ni / g.dpt, &g.per_sm);
    if (e == cudaSuccess && g.per_sm < 1) e = cudaErrorInvalidConfiguration;
    if (e == cudaSuccess) e = cudaEventCreate(&g.ev0);
    if (e == cudaSuccess) e = cudaEventCreate(&g.ev1);
    if (e != cudaSuccess) {
      if (g.ev0) cudaEventDestroy(g.ev0);
      lb_rt_destroy(h);
      return bcuda(b, e, "batched kernel occupancy");
    }
    for (int z : kZCandidates) g.cands.push_back(z);
    g.cost.assign(g.cands.size() + 1, 0.0);  // z chunks, then the alternative kernel
    g.alt_zc = batch_alt_zc(c.storage, g.dpt);
    if (g.alt_zc &&
        (occupancy_static_batch(c.storage, g.dpt, g.alt_zc, g.Ni / g.dpt, &g.alt_per_sm, 1) !=
             cudaSuccess ||
         g.alt_per_sm < 1)) {
      (void)cudaGetLastError();
      g.alt_zc = 0;
    }
    if (!b->cfg.autotune) g.tuned = true;
    b->groups.push_back(g);
    gi = (int)b->groups.size() - 1;
  }
  cudaEvent_t ready = nullptr;
  cudaError_t er = cudaEventCreateWithFlags(&ready, cudaEventDisableTiming);
  if (er == cudaSuccess) er = cudaEventRecord(ready, h->stream);
  if (er != cudaSuccess) {
    if (ready) cudaEventDestroy(ready);
    lb_rt_destroy(h);
    return bcuda(b, er, "admission event");
  }
  Member& m = b->slots[s];
  m.h = h;
  m.nsteps = nsteps;
  m.bytes = bytes;
  m.group = gi;
  m.used = true;
  m.ready = ready;
  m.joined = false;
  m.done_tick = -1;
  b->used += bytes;
  // a problem with fewer planes than the alternative kernel's batch keeps
  // its group on the plan's own kernel
  Group& grp = b->groups[gi];
  if (grp.alt_zc && h->grid.nz < grp.alt_zc) {
    grp.alt_zc = 0;
    grp.alt = 0;
    if (grp.stage == 1) {
      grp.stage = 0;
      grp.tuned = true;
    }
  }
  // tensor maps of both parities (for the alternative kernel too, whose
  // boxes hold its planes per batch), copied to the device array at the
  // next tick
  for (int par = 0; par < 2; ++par) {
    CUtensorMap* mp = b->h_maps + (size_t)s * 8 + par * 2;
    mp[0] = h->tmap[par];
    if (c.storage != LB_RT_F32) mp[1] = h->emap[par];
    if (grp.alt_zc) {
      std::string terr;
      const bool ok = c.storage == LB_RT_F32
                          ? make_pop_tensor_map(mp + 4, h->grid, h->Ni, h->pop[par], h->dpt,
                                                grp.alt_zc, terr)
                          : make_pop16_tensor_map(mp + 4, h->grid, h->Ni, h->pop[par], c.storage,
                                                  h->dpt, grp.alt_zc, terr) &&
                                make_e_tensor_map(mp + 5, h->grid, h->ef[par], grp.alt_zc, terr);
      if (!ok) {
        m = Member{};
        b->used -= bytes;
        cudaEventDestroy(ready);
        lb_rt_destroy(h);
        return bfail(b, LB_RT_ECUDA, "tensor maps: " + terr);
      }
    }
  }
  b->maps_dirty = true;
  *slot = s;
  return LB_RT_OK;
}

lb_rt_status lb_rt_batch_tick(lb_rt_batch* b, int* n_active) {
  if (!b) return LB_RT_EINVAL;
  const int K = b->cfg.steps_per_tick;
  const int G = (int)b->groups.size();
  const long long t = b->ticks;
  const int buf = (int)(t & 1);
  // tick t - 2 read the staging tables of this parity: wait for it (and
  // for nothing later)
  if (t >= 2) BCK(b, cudaEventSynchronize(b->tick_ev[(t - 2) % lb_rt_batch::kTickEvents]));
  // plan[k][g]: slots of group g that take step k of this tick
  std::vector<std::vector<std::vector<int>>> plan(K, std::vector<std::vector<int>>(G));
  int active = 0;
  std::vector<long long> group_sd(G, 0);
  for (int s = 0; s < (int)b->slots.size(); ++s) {
    const Member& m = b->slots[s];
    if (!m.used) continue;
    const long long rem = m.nsteps - m.h->steps;
    if (rem <= 0) continue;
    ++active;
    const long long take = std::min<long long>(rem, K);
    for (int k = 0; k < take; ++k) plan[k][m.group].push_back(s);
    group_sd[m.group] += take * m.h->grid.sites;
  }
  if (n_active) *n_active = active;
  if (!active) return LB_RT_OK;
  // autotuner: a group whose member sites changed by more than 2x is retuned
  bool tuning = false;
  for (int g = 0; g < G; ++g) {
    Group& gr = b->groups[g];
    if (!group_sd[g]) continue;
    long long sites = 0;
    for (int s : plan[0][g]) sites += b->slots[s].h->grid.sites;
    if (b->cfg.autotune && gr.tuned &&
        (sites > 2 * gr.tuned_sites || 2 * sites < gr.tuned_sites)) {
      gr.tuned = false;
      gr.cand = 0;
      gr.stage = 0;
    }
    if (!gr.tuned) {
      if (gr.stage == 0) {
        gr.zchunk = gr.cands[gr.cand];
        gr.alt = 0;
        if (gr.cand == 0) gr.tuned_sites = sites;
      } else {
        gr.alt = 1;  // the alternative kernel at the best z chunk
      }
      tuning = true;
    }
  }
  // pairing: exactly two groups with steps in this tick whose tile plans
  // have a paired kernel share one launch per step (mode 1), or do so when
  // the autotuner measured it faster (mode 2); never while z chunks are tuned
  int pa = -1, pb = -1;
  if (b->cfg.pair_groups && !tuning) {
    std::vector<int> act;
    for (int g = 0; g < G; ++g)
      if (group_sd[g]) act.push_back(g);
    if (act.size() == 2) {
      const Group& g0 = b->groups[act[0]];
      const Group& g1 = b->groups[act[1]];
      const int st = b->cfg.storage;
      if (static_batch_pair_supported(st, g0.dpt, g0.zc_now(), g1.dpt, g1.zc_now())) {
        pa = act[0];
        pb = act[1];
      } else if (static_batch_pair_supported(st, g1.dpt, g1.zc_now(), g0.dpt, g0.zc_now())) {
        pa = act[1];
        pb = act[0];
      }
    }
  }
  if (pa >= 0 && (pa != b->pair_a || pb != b->pair_b)) {
    const Group& A = b->groups[pa];
    const Group& B = b->groups[pb];
    int per_sm = 0;
    cudaError_t e = occupancy_static_batch_pair(b->cfg.storage, A.dpt, A.zc_now(), A.Ni / A.dpt,
                                                B.dpt, B.zc_now(), B.Ni / B.dpt, &per_sm);
    if (e != cudaSuccess) return bcuda(b, e, "paired kernel occupancy");
    b->pair_a = pa;
    b->pair_b = pb;
    b->pair_per_sm = per_sm;
    b->pair_choice = -1;
    b->pair_trial = 0;
  }
  if (pa >= 0 && b->pair_per_sm < 1) pa = pb = -1;
  bool pair_timed = false;  // this tick is one of mode 2's two trials
  if (pa >= 0 && b->cfg.pair_groups == 2) {
    // timed again when the pair's sites have changed by more than 2x
    long long sites = 0;
    for (int g : {pa, pb})
      for (int s : plan[0][g]) sites += b->slots[s].h->grid.sites;
    if (b->pair_choice >= 0 && (sites > 2 * b->pair_sites || 2 * sites < b->pair_sites)) {
      b->pair_choice = -1;
      b->pair_trial = 0;
    }
    if (b->pair_choice < 0 && b->pair_trial == 0) b->pair_sites = sites;
    if (b->pair_choice < 0) {
      pair_timed = true;
      if (b->pair_trial == 0) pa = pb = -1;  // first trial: separate launches
    } else if (b->pair_choice == 0) {
      pa = pb = -1;
    }
  }
  // descriptor tables [step][group members]
  size_t ndesc = 0;
  for (int k = 0; k < K; ++k)
    for (int g = 0; g < G; ++g) ndesc += plan[k][g].size();
  if (ndesc > b->desc_cap[buf]) {
    cudaFreeHost(b->h_desc[buf]);
    cudaFree(b->d_desc[buf]);
    b->h_desc[buf] = nullptr;
    b->d_desc[buf] = nullptr;
    b->desc_cap[buf] = 0;
    b->graph_sig[buf].clear();  // a captured graph refers to the old tables
    if (b->exec[buf]) cudaGraphExecDestroy(b->exec[buf]);
    if (b->graph[buf]) cudaGraphDestroy(b->graph[buf]);
    b->exec[buf] = nullptr;
    b->graph[buf] = nullptr;
    const size_t cap = std::max<size_t>(ndesc, 2 * b->slots.size());
    BCK(b, cudaMallocHost((void**)&b->h_desc[buf], sizeof(ProblemDesc) * cap));
    BCK(b, cudaMalloc((void**)&b->d_desc[buf], sizeof(ProblemDesc) * cap));
    b->desc_cap[buf] = cap;
  }
  ProblemDesc* h_desc = b->h_desc[buf];
  ProblemDesc* d_desc = b->d_desc[buf];
  std::vector<Launch> launches;
  std::vector<long long> sig;
  sig.push_back((long long)ndesc);
  size_t at = 0;
  for (int k = 0; k < K; ++k) {
    const size_t first_of_step = launches.size();
    for (int g = 0; g < G; ++g) {
      const auto& ms = plan[k][g];
      if (ms.empty()) continue;
      const Group& gr = b->groups[g];
      Launch L{g, (int)at, (int)ms.size(), 0, 0};
      for (int s : ms) {
        const lb_rt* h = b->slots[s].h;
        const int cur = (int)((h->cur + k) & 1);
        ProblemDesc& d = h_desc[at++];
        d = ProblemDesc{};
        d.g = h->grid;
        d.out = h->pop[cur ^ 1];
        d.e_out = h->ef[cur ^ 1];
        d.tmap = b->d_maps + (size_t)s * 8 + gr.alt * 4 + cur * 2;
        d.emap = b->d_maps + (size_t)s * 8 + gr.alt * 4 + cur * 2 + 1;
        d.cf = h->sc;
        d.dt = (float)h->dt;
        d.collision = h->cfg.collision;
        d.lambda_iters = h->cfg.lambda_iters;
        d.nzc = std::max(1, std::min(h->grid.nz, (h->grid.nz + gr.zchunk - 1) / gr.zchunk));
        d.tile_start = L.ntiles;
        d.ntiles = (h->grid.nx + 63) / 64 * h->grid.ny * d.nzc;
        d.budget_partials = nullptr;
        L.ntiles += d.ntiles;
        L.sd += h->grid.sites * (long long)gr.Ni;
        if (h->grid.periodic[0] || h->grid.periodic[1] || h->grid.periodic[2]) L.periodic = 1;
        sig.push_back(s);
        sig.push_back(d.nzc);
      }
      launches.push_back(L);
    }
    // both groups of the pair step at k: one launch, CTAs split so that
    // both halves take about as long (site-direction updates per warp)
    if (pa >= 0 && launches.size() == first_of_step + 2) {
      Launch& L0 = launches[first_of_step];
      const Launch L1 = launches[first_of_step + 1];
      Launch A = L0.group == pa ? L0 : L1;
      const Launch& Bl = L0.group == pa ? L1 : L0;
      const Group& GA = b->groups[pa];
      const Group& GB = b->groups[pb];
      long long S = std::min<long long>((long long)b->pair_per_sm * b->sms,
                                        (long long)A.ntiles + Bl.ntiles);
      if (S >= 2) {
        const double wa = (double)A.sd / (GA.Ni / GA.dpt), wb = (double)Bl.sd / (GB.Ni / GB.dpt);
        long long ca = std::llround((double)S * wa / (wa + wb));
        ca = std::max<long long>(1, std::min<long long>(ca, S - 1));
        ca = std::min<long long>(ca, A.ntiles);
        ca = std::max<long long>(ca, S - Bl.ntiles);
        A.b_group = Bl.group;
        A.b_first = Bl.first;
        A.b_nprob = Bl.nprob;
        A.b_ntiles = Bl.ntiles;
        A.b_periodic = Bl.periodic;
        A.b_sd = Bl.sd;
        A.ctas_a = (int)ca;
        A.ctas = (int)S;
        launches.resize(first_of_step);
        launches.push_back(A);
      }
    }
    for (size_t i = first_of_step; i < launches.size(); ++i) {
      const Launch& L = launches[i];
      for (long long v : {(long long)L.group, (long long)b->groups[L.group].alt,
                          (long long)L.first, (long long)L.nprob,
                          (long long)L.ntiles, (long long)L.periodic, (long long)L.b_group,
                          (long long)L.b_first, (long long)L.b_nprob, (long long)L.b_ntiles,
                          (long long)L.ctas_a, (long long)L.ctas})
        sig.push_back(v);
    }
  }
  // problems stepped for the first time: their admission (initial state,
  // fields) ran on their own streams
  for (int s = 0; s < (int)b->slots.size(); ++s) {
    Member& m = b->slots[s];
    if (!m.used || m.joined || m.nsteps - m.h->steps <= 0) continue;
    BCK(b, cudaStreamWaitEvent(b->stream, m.ready, 0));
    m.joined = true;
  }
  // the tick's device work: table uploads, then the launches (per group when
  // the z-chunk autotuner times groups, in step order otherwise)
  auto enqueue = [&](bool timed) -> cudaError_t {
    cudaError_t e = cudaSuccess;
    if (b->maps_dirty || !timed)
      e = cudaMemcpyAsync(b->d_maps, b->h_maps, sizeof(CUtensorMap) * 8 * b->slots.size(),
                          cudaMemcpyHostToDevice, b->stream);
    if (e == cudaSuccess)
      e = cudaMemcpyAsync(d_desc, h_desc, sizeof(ProblemDesc) * ndesc, cudaMemcpyHostToDevice,
                          b->stream);
    auto batch_of = [&](int g, int first, int nprob, int ntiles, int periodic, int ctas) {
      const Group& gr = b->groups[g];
      BatchLaunch B{};
      B.table = d_desc + first;
      B.nprob = nprob;
      B.ntiles = ntiles;
      B.N = gr.Ni;
      B.dpt = gr.dpt;
      B.zc = gr.zc_now();
      B.alt = gr.alt;
      B.storage = b->cfg.storage;
      B.ctas = ctas;
      B.periodic = periodic;
      B.err = b->d_err;
      return B;
    };
    auto single = [&](const Launch& L) -> cudaError_t {
      Group& gr = b->groups[L.group];
      const int per_sm = gr.alt ? gr.alt_per_sm : gr.per_sm;
      const int ctas = (int)std::min<long long>((long long)per_sm * b->sms, L.ntiles);
      gr.last_zc = gr.zc_now();
      gr.ctas = ctas;
      gr.paired = false;
      return launch_tma_static_batch(batch_of(L.group, L.first, L.nprob, L.ntiles, L.periodic, ctas),
                                     gr.table, b->stream);
    };
    if (timed && tuning) {
      for (int g = 0; g < G && e == cudaSuccess; ++g) {
        Group& gr = b->groups[g];
        const bool time_it = !gr.tuned && group_sd[g] > 0;
        if (time_it) e = cudaEventRecord(gr.ev0, b->stream);
        for (const Launch& L : launches)
          if (L.group == g && e == cudaSuccess) e = single(L);
        if (e == cudaSuccess && time_it) e = cudaEventRecord(gr.ev1, b->stream);
      }
      return e;
    }
    if (e == cudaSuccess && timed) e = cudaEventRecord(b->pev0, b->stream);
    for (const Launch& L : launches) {
      if (e != cudaSuccess) break;
      if (L.b_group < 0) {
        e = single(L);
        continue;
      }
      Group& ga = b->groups[L.group];
      Group& gb = b->groups[L.b_group];
      const BatchLaunch A = batch_of(L.group, L.first, L.nprob, L.ntiles, L.periodic, L.ctas_a);
      const BatchLaunch B =
          batch_of(L.b_group, L.b_first, L.b_nprob, L.b_ntiles, L.b_periodic, L.ctas - L.ctas_a);
      ga.ctas = L.ctas_a;
      gb.ctas = L.ctas - L.ctas_a;
      ga.last_zc = ga.zc_now();
      gb.last_zc = gb.zc_now();
      ga.paired = gb.paired = true;
      e = launch_static_batch_pair(A, ga.table, B, gb.table, L.ctas_a, L.ctas, b->stream);
    }
    if (e == cudaSuccess && timed) e = cudaEventRecord(b->pev1, b->stream);
    return e;
  };
  cudaError_t e = cudaSuccess;
  if (tuning || pair_timed || !b->cfg.use_graph) {
    e = enqueue(tuning || pair_timed);
  } else if (sig != b->graph_sig[buf] || !b->exec[buf]) {
    // capture the new plan; update the instantiated graph of this parity in
    // place where the update applies (same launches, new parameters), else
    // instantiate it afresh
    cudaGraph_t g = nullptr;
    e = cudaStreamBeginCapture(b->stream, cudaStreamCaptureModeThreadLocal);
    if (e == cudaSuccess) {
      const cudaError_t e2 = enqueue(false);
      e = cudaStreamEndCapture(b->stream, &g);
      if (e == cudaSuccess) e = e2;
    }
    bool updated = false;
    if (e == cudaSuccess && b->exec[buf]) {
      cudaGraphExecUpdateResultInfo info{};
      updated = cudaGraphExecUpdate(b->exec[buf], g, &info) == cudaSuccess;
      if (!updated) {
        (void)cudaGetLastError();
        cudaGraphExecDestroy(b->exec[buf]);
        b->exec[buf] = nullptr;
      }
    }
    if (e == cudaSuccess && !updated) e = cudaGraphInstantiate(&b->exec[buf], g, 0);
    if (b->graph[buf]) cudaGraphDestroy(b->graph[buf]);
    b->graph[buf] = g;
    if (e == cudaSuccess) b->graph_sig[buf] = sig;
    else b->graph_sig[buf].clear();
    if (e == cudaSuccess) e = cudaGraphLaunch(b->exec[buf], b->stream);
  } else {
    e = cudaGraphLaunch(b->exec[buf], b->stream);
  }
  if (e == cudaSuccess) e = cudaEventRecord(b->tick_ev[t % lb_rt_batch::kTickEvents], b->stream);
  if (e != cudaSuccess) return bcuda(b, e, "batch tick");
  b->maps_dirty = false;
  b->ticks = t + 1;
  // the members' step counters, buffer parity and, for those that finish
  // in this tick, the tick to wait for
  for (int s = 0; s < (int)b->slots.size(); ++s) {
    Member& m = b->slots[s];
    if (!m.used) continue;
    const long long rem = m.nsteps - m.h->steps;
    if (rem <= 0) continue;
    const long long take = std::min<long long>(rem, K);
    m.h->cur ^= (int)(take & 1);
    m.h->steps += take;
    if (m.h->steps >= m.nsteps) m.done_tick = t;
  }
  if (pair_timed) {
    BCK(b, cudaStreamSynchronize(b->stream));
    float ms = 0.f;
    BCK(b, cudaEventElapsedTime(&ms, b->pev0, b->pev1));
    long long sd = 0;
    for (int g = 0; g < G; ++g) sd += group_sd[g] * b->groups[g].Ni;
    b->pair_cost[b->pair_trial] = sd ? ms / (double)sd : 0.0;
    if (++b->pair_trial == 2) b->pair_choice = b->pair_cost[1] < b->pair_cost[0] ? 1 : 0;
  }
  if (tuning) {
    BCK(b, cudaStreamSynchronize(b->stream));
    for (int g = 0; g < G; ++g) {
      Group& gr = b->groups[g];
      if (gr.tuned || !group_sd[g]) continue;
      float ms = 0.f;
      BCK(b, cudaEventElapsedTime(&ms, gr.ev0, gr.ev1));
      const int nz = (int)gr.cands.size();
      if (gr.stage == 1) {
        // keep the alternative kernel only if it beat the best z chunk
        gr.cost[nz] = ms / (double)group_sd[g];
        double best = gr.cost[0];
        for (int i = 1; i < nz; ++i) best = std::min(best, gr.cost[i]);
        gr.alt = gr.cost[nz] < best ? 1 : 0;
        gr.stage = 0;
        gr.tuned = true;
        continue;
      }
      gr.cost[gr.cand] = ms / (double)group_sd[g];
      if (++gr.cand == nz) {
        int best = 0;
        for (int i = 1; i < nz; ++i)
          if (gr.cost[i] < gr.cost[best]) best = i;
        gr.zchunk = gr.cands[best];
        if (gr.alt_zc) {
          gr.stage = 1;
        } else {
          gr.tuned = true;
        }
      }
    }
  }
  return LB_RT_OK;
}

lb_rt_status lb_rt_batch_sync(lb_rt_batch* b) {
  if (!b) return LB_RT_EINVAL;
  BCK(b, cudaStreamSynchronize(b->stream));
  flush_grave(b);  // nothing is in flight: released memory goes back now
  unsigned word = 0;
  BCK(b, cudaMemcpy(&word, b->d_err, sizeof(unsigned), cudaMemcpyDeviceToHost));
  if (word) return bfail(b, LB_RT_ETIMEDOUT, "device error word set by a batched step");
  return LB_RT_OK;
}

lb_rt_status lb_rt_batch_poll(lb_rt_batch* b, int* slots, int max, int* n) {
  if (!b) return LB_RT_EINVAL;
  if (!n || (max > 0 && !slots)) return bfail(b, LB_RT_EINVAL, "bad poll arguments");
  int c = 0;
  for (int s = 0; s < (int)b->slots.size(); ++s) {
    const Member& m = b->slots[s];
    if (m.used && m.h->steps >= m.nsteps && tick_done(b, m.done_tick)) {
      if (c < max) slots[c] = s;
      ++c;
    }
  }
  *n = std::min(c, max);
  return LB_RT_OK;
}

lb_rt_status lb_rt_batch_moments(lb_rt_batch* b, int slot, float* E, float* F, float* P,
                                 int ptr_kind) {
  if (!b) return LB_RT_EINVAL;
  if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used)
    return bfail(b, LB_RT_EINVAL, "bad slot");
  // the problem's ticks have to be complete (its own stream does not see them)
  if (b->ticks > 0)
    BCK(b, cudaEventSynchronize(b->tick_ev[(b->ticks - 1) % lb_rt_batch::kTickEvents]));
  lb_rt* h = b->slots[slot].h;
  const lb_rt_status st = lb_rt_moments(h, E, F, P, nullptr, ptr_kind);
  if (st != LB_RT_OK) return bfail(b, st, lb_rt_last_error(h));
  return LB_RT_OK;
}

lb_rt_status lb_rt_batch_steps(const lb_rt_batch* b, int slot, long long* steps) {
  if (!b || !steps || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used)
    return LB_RT_EINVAL;
  *steps = b->slots[slot].h->steps;
  return LB_RT_OK;
}

lb_rt_status lb_rt_batch_release(lb_rt_batch* b, int slot) {
  if (!b) return LB_RT_EINVAL;
  if (slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used)
    return bfail(b, LB_RT_EINVAL, "bad slot");
  Member& m = b->slots[slot];
  // its last tick may still run: the memory goes back at the next
  // synchronisation (or when an admission needs it)
  b->grave.push_back(m.h);
  b->grave_bytes += m.bytes;
  if (m.ready) cudaEventDestroy(m.ready);
  m = Member{};
  return LB_RT_OK;
}

lb_rt_status lb_rt_batch_plan(const lb_rt_batch* b, int slot, int* dirs_per_warp,
                              int* planes_per_batch, int* paired) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used) return LB_RT_EINVAL;
  const Group& g = b->groups[b->slots[slot].group];
  if (dirs_per_warp) *dirs_per_warp = g.dpt;
  if (planes_per_batch) *planes_per_batch = g.last_zc ? g.last_zc : g.zc_now();
  if (paired) *paired = g.paired ? 1 : 0;
  return LB_RT_OK;
}

lb_rt_status lb_rt_batch_tuning(const lb_rt_batch* b, int slot, int* zchunk, int* ctas) {
  if (!b || slot < 0 || slot >= (int)b->slots.size() || !b->slots[slot].used) return LB_RT_EINVAL;
  const Group& g = b->groups[b->slots[slot].group];
  if (zchunk) *zchunk = g.zchunk;
  if (ctas) *ctas = g.ctas;
  return LB_RT_OK;
}

const char* lb_rt_batch_last_error(const lb_rt_batch* b) { return b ? b->msg.c_str() : ""; }

}  // extern "C"
