// amh_api.cu -- the C ABI declared in include/amh.h: argument checks, device
// memory, launch configuration (with a small autotuner) and the calls that
// run the kernels of amh_global.cu, amh_local.cu and amh_misc.cu.
#include <algorithm>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <string>
#include <vector>

#include "amh.h"
#include "amh_internal.h"

using namespace amh;

struct amh_ctx {
  int device = 0;
  int precision = 32;
  amh_options opt;
  cudaStream_t stream = nullptr;
  int nprot = 0;
  std::vector<int> L, nch;
  std::vector<ProteinDev> prot_h;
  std::vector<long long> t_host;  // per protein proposal counter (mirror)
  int total_chains = 0;
  long long tors_total = 0;
  int Lmax = 0, nmax = 0;
  int B = 0, Bp = 0;
  double c0 = 0, w = 0;
  long long rows_total = 0;
  // device memory
  void* table = nullptr;
  void* theta = nullptr;
  void* best_theta = nullptr;
  float* f32buf = nullptr;  // FP32 staging for precision-64 conversions
  long long* tcount = nullptr;
  void* coords = nullptr;  // per chain C-betas (keep_coords), precision R
  double* E_cur = nullptr;
  double* best_E = nullptr;
  long long* acc = nullptr;
  ProteinDev* prot_d = nullptr;
  int* chain_prot_d = nullptr;
  GroupDev* ggroups_d = nullptr;  // global groups for the chosen C
  int nggroups = 0;
  GroupDev* lgroups_d[6] = {nullptr, nullptr, nullptr, nullptr, nullptr, nullptr};  // Gc = 1..32
  int nlgroups[6] = {0, 0, 0, 0, 0, 0};
  int* queue = nullptr;
  int* err = nullptr;
  unsigned long long* pair_count = nullptr;  // global sweeps' straddle terms: [0] formed, [1] read
  double* tcache = nullptr;  // the global sweeps' rebuild scratch (SweepArgs::tcache)
  size_t tcache_bytes = 0;
  TraceRec* trace = nullptr;
  long long* trace_count = nullptr;
  // launch configuration
  int C = 8, threads = 256, grid_global = 1;
  // chain groups (FP32 far-field kernel): chains per CTA, warps per chain, grid
  bool use_warp = false;
  int warpW = 4, warpG = 1, grid_warp = 1;
  GroupDev* wgroups_d = nullptr;  // one chain per group
  int nwgroups = 0;
  int stage_depth = 0;  // > 0: global sweeps stage table rows through shared memory
  cudaTextureObject_t tex = 0;  // FP32 table as a 1-D texture (0: not used)
  double* ladder = nullptr;  // parallel tempering: per-slot temperature factors
  int ladder_K = 0;
  unsigned long long xround = 0;  // exchange rounds so far (Philox counter)
  int sm_count = 1;
  size_t smem_optin = 0;
  std::string msg;
  bool broken = false;
  // E_cur is owed a recomputation: the state was replaced (amh_set_state,
  // amh_noisy_restart) and no global sweep or energy call has run since
  bool energy_stale = false;
};

namespace {

// room left for the kernels' static shared memory when sizing dynamic smem
constexpr size_t kStaticSmemMargin = 1024;

thread_local std::string g_free_error;

amh_status set_err(amh_ctx* ctx, amh_status st, const std::string& m) {
  if (ctx) {
    ctx->msg = m;
    // a device error, or a bounded wait that gave up part-way through a
    // sweep, leaves the chains' state undefined
    if (st == AMH_ECUDA || st == AMH_ETIMEOUT) ctx->broken = true;
  } else {
    g_free_error = m;
  }
  return st;
}

amh_status cuda_fail(amh_ctx* ctx, cudaError_t e, const char* what) {
  std::string m = std::string(what) + ": " + cudaGetErrorString(e);
  if (e == cudaErrorMemoryAllocation) {
    cudaGetLastError();
    if (ctx) ctx->msg = m;
    return AMH_ENOMEM;
  }
  return set_err(ctx, AMH_ECUDA, m);
}

#define CK(ctx, call)                                         \
  do {                                                        \
    cudaError_t e_ = (call);                                  \
    if (e_ != cudaSuccess) return cuda_fail((ctx), e_, #call); \
  } while (0)

bool is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <class R>
Tab<R> make_tab(const amh_ctx* ctx) {
  Tab<R> t;
  t.E = (const typename Vec2<R>::T*)ctx->table;
  t.inv_w = (R)(1.0 / ctx->w);
  t.off = (R)(-ctx->c0 / ctx->w);
  t.umax = (R)(ctx->B - 1);
  t.k1 = (R)(1.0 / ctx->w / (ctx->B - 1));
  t.k2 = (R)(-ctx->c0 / ctx->w / (ctx->B - 1));
  t.Bp = ctx->Bp;
  t.tex = ctx->tex;
  return t;
}

template <class R>
SweepArgs<R> make_args(amh_ctx* ctx) {
  SweepArgs<R> a;
  memset(&a, 0, sizeof(a));
  a.prot = ctx->prot_d;
  a.groups = ctx->ggroups_d;
  a.ngroups = ctx->nggroups;
  a.queue = ctx->queue;
  a.theta = (R*)ctx->theta;
  a.best_theta = (R*)ctx->best_theta;
  a.tcount = ctx->tcount;
  a.E_cur = ctx->E_cur;
  a.best_E = ctx->best_E;
  a.acc_out = ctx->acc;
  a.tab = make_tab<R>(ctx);
  a.geom = ideal_geometry<R>();
  a.geom64 = ideal_geometry<double>();
  a.resync_every = ctx->opt.resync_every;
  a.lattice_K = ctx->opt.lattice_K;
  a.Lmax = ctx->Lmax;
  a.nmax = ctx->nmax;
  a.trace = ctx->trace;
  a.trace_chains = ctx->trace ? ctx->opt.trace_chains : 0;
  a.trace_cap = ctx->opt.trace_capacity;
  a.trace_count = ctx->trace_count;
  a.err = ctx->err;
  a.coords = (R*)ctx->coords;
  a.wait_test = ctx->opt.wait_test;
  a.stage_depth = ctx->stage_depth;
  // last bin centre c0 + (B-1) w: beyond it sat(d k1 + k2) = 1 and the FP32
  // term is the constant last entry; 0.01 A covers the rounding of the
  // distances and of the bounding spheres (~1e-5 A)
  // the chunks of a fixed side are bits of one word
  a.far_skip = ctx->precision == 32 && ctx->opt.far_pairs == 0 &&
               ctx->Lmax <= kMaxChunks * kPairChunk + 1;
  a.far_cut = (float)(ctx->c0 + (ctx->B - 1) * ctx->w + 0.01);
  a.pair_count = ctx->pair_count;
  a.tcache = ctx->tcache;
  a.ladder = ctx->ladder_K ? ctx->ladder : nullptr;
  a.ladder_K = ctx->ladder_K;
  return a;
}

// ---- dispatch over (precision, C, staging) ---------------------------------
int row_bytes(const amh_ctx* ctx) { return ctx->Bp * (ctx->precision == 64 ? 16 : 8); }

template <class R>
size_t gsmem(int C, int Lmax, int nmax, int threads, int D, int RB) {
  switch (C) {
    case 1: return global_smem_bytes<R, 1>(Lmax, nmax, threads, D, RB);
    case 2: return global_smem_bytes<R, 2>(Lmax, nmax, threads, D, RB);
    case 4: return global_smem_bytes<R, 4>(Lmax, nmax, threads, D, RB);
    default: return global_smem_bytes<R, 8>(Lmax, nmax, threads, D, RB);
  }
}
template <>
size_t gsmem<double>(int C, int Lmax, int nmax, int threads, int D, int RB) {
  switch (C) {
    case 1: return global_smem_bytes<double, 1>(Lmax, nmax, threads, D, RB);
    case 2: return global_smem_bytes<double, 2>(Lmax, nmax, threads, D, RB);
    default: return global_smem_bytes<double, 4>(Lmax, nmax, threads, D, RB);
  }
}

template <class R>
cudaError_t gset(int C, size_t bytes) {
  cudaError_t e = cudaSuccess;
  switch (C) {
    case 1: return global_set_smem<R, 1, false>(bytes);
    case 2: return global_set_smem<R, 2, false>(bytes);
    case 4:
      e = global_set_smem<R, 4, false>(bytes);
      return e != cudaSuccess ? e : global_set_smem<R, 4, true>(bytes);
    default:
      e = global_set_smem<R, 8, false>(bytes);
      return e != cudaSuccess ? e : global_set_smem<R, 8, true>(bytes);
  }
}
template <>
cudaError_t gset<double>(int C, size_t bytes) {
  switch (C) {
    case 1: return global_set_smem<double, 1, false>(bytes);
    case 2: return global_set_smem<double, 2, false>(bytes);
    default: return global_set_smem<double, 4, false>(bytes);
  }
}

template <class R>
cudaError_t gocc(int C, bool ST, int threads, size_t sm, int* per_sm) {
  switch (C) {
    case 1: return global_occupancy<R, 1, false>(threads, sm, per_sm);
    case 2: return global_occupancy<R, 2, false>(threads, sm, per_sm);
    case 4: return ST ? global_occupancy<R, 4, true>(threads, sm, per_sm)
                      : global_occupancy<R, 4, false>(threads, sm, per_sm);
    default: return ST ? global_occupancy<R, 8, true>(threads, sm, per_sm)
                       : global_occupancy<R, 8, false>(threads, sm, per_sm);
  }
}
template <>
cudaError_t gocc<double>(int C, bool ST, int threads, size_t sm, int* per_sm) {
  (void)ST;
  switch (C) {
    case 1: return global_occupancy<double, 1, false>(threads, sm, per_sm);
    case 2: return global_occupancy<double, 2, false>(threads, sm, per_sm);
    default: return global_occupancy<double, 4, false>(threads, sm, per_sm);
  }
}

template <class R>
cudaError_t glaunch(bool energy, int C, bool ST, const SweepArgs<R>& a, int threads, int grid,
                    cudaStream_t st) {
  switch (C) {
    case 1: return energy ? launch_energy<R, 1>(a, threads, grid, st)
                          : launch_global<R, 1, false>(a, threads, grid, st);
    case 2: return energy ? launch_energy<R, 2>(a, threads, grid, st)
                          : launch_global<R, 2, false>(a, threads, grid, st);
    case 4:
      if (energy) return launch_energy<R, 4>(a, threads, grid, st);
      return ST ? launch_global<R, 4, true>(a, threads, grid, st)
                : launch_global<R, 4, false>(a, threads, grid, st);
    default:
      if (energy) return launch_energy<R, 8>(a, threads, grid, st);
      return ST ? launch_global<R, 8, true>(a, threads, grid, st)
                : launch_global<R, 8, false>(a, threads, grid, st);
  }
}
template <>
cudaError_t glaunch<double>(bool energy, int C, bool ST, const SweepArgs<double>& a, int threads,
                            int grid, cudaStream_t st) {
  (void)ST;
  switch (C) {
    case 1: return energy ? launch_energy<double, 1>(a, threads, grid, st)
                          : launch_global<double, 1, false>(a, threads, grid, st);
    case 2: return energy ? launch_energy<double, 2>(a, threads, grid, st)
                          : launch_global<double, 2, false>(a, threads, grid, st);
    default: return energy ? launch_energy<double, 4>(a, threads, grid, st)
                           : launch_global<double, 4, false>(a, threads, grid, st);
  }
}

int max_C(int precision) { return precision == 64 ? 4 : 8; }

// Group chains of each protein C at a time; order groups by decreasing cost
// (a global sweep of a chain costs ~ L^3) so the persistent CTAs that pull
// from the queue finish together.
std::vector<GroupDev> make_groups(const amh_ctx* ctx, int C) {
  std::vector<GroupDev> g;
  for (int p = 0; p < ctx->nprot; ++p) {
    for (int c = 0; c < ctx->nch[p]; c += C) {
      GroupDev d;
      d.protein = p;
      d.chain0 = ctx->prot_h[p].chain0 + c;
      d.nchains = std::min(C, ctx->nch[p] - c);
      d.pad = 0;
      g.push_back(d);
    }
  }
  std::stable_sort(g.begin(), g.end(), [&](const GroupDev& a, const GroupDev& b) {
    return ctx->L[a.protein] > ctx->L[b.protein];
  });
  return g;
}

amh_status upload_groups(amh_ctx* ctx, const std::vector<GroupDev>& g, GroupDev** dst, int* n) {
  if (*dst) {
    cudaFree(*dst);
    *dst = nullptr;
  }
  CK(ctx, cudaMalloc(dst, sizeof(GroupDev) * std::max<size_t>(1, g.size())));
  CK(ctx, cudaMemcpy(*dst, g.data(), sizeof(GroupDev) * g.size(), cudaMemcpyHostToDevice));
  *n = (int)g.size();
  return AMH_OK;
}

// Deepest staging ring (slots per warp, 2..4) that fits, or 0.  Staging
// exists for FP32 with 4 or 8 chains per CTA.
int stage_depth_for(const amh_ctx* ctx, int C, int threads) {
  if (ctx->precision != 32 || (C != 4 && C != 8)) return 0;
  for (int D = 4; D >= 2; --D)
    if (gsmem<float>(C, ctx->Lmax, ctx->nmax, threads, D, row_bytes(ctx)) <= ctx->smem_optin - kStaticSmemMargin)
      return D;
  return 0;
}

template <class R>
amh_status configure_global(amh_ctx* ctx, int C, int threads, int D) {
  const size_t sm = gsmem<R>(C, ctx->Lmax, ctx->nmax, threads, D, D ? row_bytes(ctx) : 0);
  if (sm > ctx->smem_optin - kStaticSmemMargin)
    return set_err(ctx, AMH_EINVAL, "shared memory for this C does not fit");
  amh_status st = upload_groups(ctx, make_groups(ctx, C), &ctx->ggroups_d, &ctx->nggroups);
  if (st) return st;
  ctx->C = C;
  ctx->threads = threads;
  ctx->stage_depth = D;
  // persistent grid: as many CTAs as are resident at once, at most one per group
  int per_sm = 1;
  CK(ctx, gocc<R>(C, D > 0, threads, sm, &per_sm));
  ctx->grid_global = std::max(1, std::min(ctx->nggroups, ctx->sm_count * std::max(per_sm, 1)));
  // the rebuild's scratch: the residue transforms of every chain slot of
  // every resident CTA (grown here, before any sweep is issued, never inside
  // a captured stream)
  const size_t need = (size_t)ctx->grid_global * C * ctx->Lmax * 12 * sizeof(double);
  if (need > ctx->tcache_bytes) {
    if (ctx->tcache) cudaFree(ctx->tcache);
    ctx->tcache = nullptr;
    ctx->tcache_bytes = 0;
    CK(ctx, cudaMalloc(&ctx->tcache, need));
    ctx->tcache_bytes = need;
  }
  return AMH_OK;
}

// The warp-per-chain kernel applies to FP32 sweeps that skip the far field
// (chunk bits of L <= 64 chunks) without staging.
bool warp_applies(const amh_ctx* ctx) {
  return ctx->precision == 32 && ctx->opt.far_pairs == 0 && ctx->opt.stage_table != 1 &&
         ctx->Lmax <= kMaxChunks * kPairChunk && ctx->opt.global_kernel != 1;
}

amh_status configure_warp(amh_ctx* ctx, int W, int G) {
  const size_t sm = gwarp_smem_bytes(ctx->Lmax, W, G);
  if (sm > ctx->smem_optin - kStaticSmemMargin || W * G > 8)
    return set_err(ctx, AMH_EINVAL, "shared memory for this many chains per CTA does not fit");
  if (!ctx->wgroups_d) {
    amh_status st = upload_groups(ctx, make_groups(ctx, 1), &ctx->wgroups_d, &ctx->nwgroups);
    if (st) return st;
  }
  int per_sm = 1;
  CK(ctx, gwarp_occupancy(W, G, sm, &per_sm));
  ctx->warpW = W;
  ctx->warpG = G;
  const int ctas = (ctx->nwgroups + W - 1) / W;
  ctx->grid_warp = std::max(1, std::min(ctas, ctx->sm_count * std::max(per_sm, 1)));
  return AMH_OK;
}

template <class R>
amh_status run_energy(amh_ctx* ctx) {
  SweepArgs<R> a = make_args<R>(ctx);
  CK(ctx, cudaMemsetAsync(ctx->queue, 0, sizeof(int), ctx->stream));
  CK(ctx, glaunch<R>(true, ctx->C, false, a, ctx->threads, ctx->grid_global, ctx->stream));
  return AMH_OK;
}

template <class R>
amh_status run_best(amh_ctx* ctx, int init) {
  CK(ctx, launch_best<R>(ctx->prot_d, ctx->chain_prot_d, ctx->total_chains, ctx->nmax,
                         (const R*)ctx->theta, (R*)ctx->best_theta, ctx->E_cur, ctx->best_E, init,
                         ctx->stream));
  return AMH_OK;
}

amh_status check_err_flag(amh_ctx* ctx) {
  int h = 0;
  CK(ctx, cudaMemcpyAsync(&h, ctx->err, sizeof(int), cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (h & 2) {
    CK(ctx, cudaMemsetAsync(ctx->err, 0, sizeof(int), ctx->stream));
    return set_err(ctx, AMH_ETIMEOUT, "a shared-memory staging wait gave up");
  }
  if (h) return set_err(ctx, AMH_ECUDA, "device reported a non-finite energy");
  return AMH_OK;
}

// Time a few global proposals around the middle of the chain for each
// candidate launch shape on scratch copies of the state; keep the fastest.
template <class R>
amh_status autotune(amh_ctx* ctx) {
  const int cand_C[4] = {1, 2, 4, 8};
  const int cand_T[4] = {64, 128, 256, 512};
  long long* t_scr = nullptr;
  R* th_scr = nullptr;
  R* bt_scr = nullptr;
  double *e_scr = nullptr, *be_scr = nullptr;
  const size_t tb = sizeof(R) * (size_t)ctx->tors_total;
  CK(ctx, cudaMalloc(&t_scr, sizeof(long long) * ctx->total_chains));
  CK(ctx, cudaMalloc(&th_scr, tb));
  CK(ctx, cudaMalloc(&bt_scr, tb));
  CK(ctx, cudaMalloc(&e_scr, sizeof(double) * ctx->total_chains));
  CK(ctx, cudaMalloc(&be_scr, sizeof(double) * ctx->total_chains));
  cudaEvent_t e0, e1;
  CK(ctx, cudaEventCreate(&e0));
  CK(ctx, cudaEventCreate(&e1));
  float best_ms = 1e30f, last_ms = 0.f;
  int bestC = 0, bestT = 256, bestD = 0;
  // three runs of up to 64 proposals, at 1/6, 1/2 and 5/6 of each sweep:
  // the straddle blocks there have the sizes a whole sweep averages over
  const long long steps = std::min(64, std::max(2, ctx->nmax / 3));
  std::vector<long long> tstart[3];
  for (int seg = 0; seg < 3; ++seg) {
    tstart[seg].resize(ctx->total_chains);
    for (int p = 0; p < ctx->nprot; ++p) {
      const long long n = ctx->prot_h[p].n;
      const long long at = std::max(0LL, n * (2 * seg + 1) / 6 - steps / 2) & ~1LL;
      for (int c = 0; c < ctx->nch[p]; ++c) tstart[seg][ctx->prot_h[p].chain0 + c] = at;
    }
  }
  // the chain-group kernel: chains per CTA and warps per chain
  int bestW = 0, bestG = 1;
  float best_warp_ms = 1e30f;
  auto time_runs = [&](auto launch) -> amh_status {
    float ms_sum = 0.f;
    for (int run = 0; run < 4; ++run) {  // run 0 warms up, runs 1-3 are timed
      const int seg = run == 0 ? 1 : run - 1;
      CK(ctx, cudaMemcpyAsync(th_scr, ctx->theta, tb, cudaMemcpyDeviceToDevice, ctx->stream));
      CK(ctx, cudaMemcpyAsync(bt_scr, ctx->theta, tb, cudaMemcpyDeviceToDevice, ctx->stream));
      CK(ctx, cudaMemcpyAsync(t_scr, tstart[seg].data(), sizeof(long long) * ctx->total_chains,
                              cudaMemcpyHostToDevice, ctx->stream));
      CK(ctx, cudaMemsetAsync(be_scr, 0x7f, sizeof(double) * ctx->total_chains, ctx->stream));
      SweepArgs<R> a = make_args<R>(ctx);
      a.theta = th_scr;
      a.best_theta = bt_scr;
      a.tcount = t_scr;
      a.E_cur = e_scr;
      a.best_E = be_scr;
      a.acc_out = nullptr;
      a.trace_chains = 0;
      a.trace_count = nullptr;
      a.coords = nullptr;
      a.wait_test = 0;
      a.pair_count = nullptr;
      a.T = 1.0;
      a.sigma = (R)0.1;
      a.seed = 12345;
      a.steps = steps;
      a.resync_every = 1 << 30;
      CK(ctx, cudaMemsetAsync(ctx->queue, 0, sizeof(int), ctx->stream));
      CK(ctx, cudaEventRecord(e0, ctx->stream));
      CK(ctx, launch(a));
      CK(ctx, cudaEventRecord(e1, ctx->stream));
      CK(ctx, cudaEventSynchronize(e1));
      float ms = 0.f;
      CK(ctx, cudaEventElapsedTime(&ms, e0, e1));
      if (run) ms_sum += ms;
    }
    last_ms = ms_sum;
    return AMH_OK;
  };
  if constexpr (sizeof(R) == 4) {
    if (warp_applies(ctx)) {
      const int candW[4] = {1, 2, 4, 8};
      const int candG[3] = {1, 2, 4};
      for (int G : candG) {
        if (ctx->opt.warps_per_chain && G != ctx->opt.warps_per_chain) continue;
        for (int W : candW) {
          if (W * G > 8 ||
              gwarp_smem_bytes(ctx->Lmax, W, G) > ctx->smem_optin - kStaticSmemMargin)
            continue;
          amh_status st = configure_warp(ctx, W, G);
          if (st) return st;
          st = time_runs([&](const SweepArgs<R>& a0) {
            SweepArgs<R> a = a0;
            a.groups = ctx->wgroups_d;
            a.ngroups = ctx->nwgroups;
            return launch_gwarp(a, W, G, ctx->grid_warp, ctx->stream);
          });
          if (st) return st;
          if (last_ms < best_warp_ms) {
            best_warp_ms = last_ms;
            bestW = W;
            bestG = G;
          }
        }
      }
    }
  }
  for (int C : cand_C) {
    if (C > max_C(ctx->precision)) continue;
    if (ctx->opt.global_kernel == 2) break;  // the CTA kernel only serves energies
    for (int T : cand_T) {
     for (int staged = 0; staged < 2; ++staged) {
      if (staged && (ctx->opt.stage_table == 2 || T < 256)) continue;
      if (!staged && ctx->opt.stage_table == 1) continue;
      const int D = staged ? stage_depth_for(ctx, C, T) : 0;
      if (staged && D == 0) continue;
      if (gsmem<R>(C, ctx->Lmax, ctx->nmax, T, D, D ? row_bytes(ctx) : 0) >
          ctx->smem_optin - kStaticSmemMargin)
        continue;
      amh_status st = configure_global<R>(ctx, C, T, D);
      if (st) return st;
      st = time_runs([&](const SweepArgs<R>& a) {
        return glaunch<R>(false, C, D > 0, a, T, ctx->grid_global, ctx->stream);
      });
      if (st) return st;
      const float ms_sum = last_ms;
      if (ms_sum < best_ms) {
        best_ms = ms_sum;
        bestC = C;
        bestT = T;
        bestD = D;
      }
     }
    }
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  cudaFree(t_scr);
  cudaFree(th_scr);
  cudaFree(bt_scr);
  cudaFree(e_scr);
  cudaFree(be_scr);
  amh_status st = check_err_flag(ctx);
  if (st) return st;
  if (bestW && (best_warp_ms <= best_ms || ctx->opt.global_kernel == 2)) {
    st = configure_warp(ctx, bestW, bestG);
    if (st) return st;
    ctx->use_warp = true;
    // energies (and a precision-64 or staged request) still use the CTA kernel
    if (!bestC) {
      bestC = 1;
      bestT = 128;
    }
  } else if (ctx->opt.global_kernel == 2) {
    return set_err(ctx, AMH_EINVAL, "the warp-per-chain kernel does not fit in shared memory");
  }
  if (!bestC) return set_err(ctx, AMH_EINVAL, "no launch shape fits in shared memory");
  return configure_global<R>(ctx, bestC, bestT, bestD);
}

template <class R>
amh_status init_impl(amh_ctx* ctx, const float* torsions, const double* table) {
  // table: p (or -ln p) -> padded R rows, via a temporary FP64 copy
  double* tmp = nullptr;
  const size_t tbytes = sizeof(double) * (size_t)ctx->rows_total * ctx->B;
  CK(ctx, cudaMalloc(&ctx->table, 2 * sizeof(R) * (size_t)ctx->rows_total * ctx->Bp + 64));
  CK(ctx, cudaMalloc(&tmp, std::max<size_t>(tbytes, 8)));
  CK(ctx, cudaMemcpy(tmp, table, tbytes, cudaMemcpyHostToDevice));
  CK(ctx, launch_prep_table<R>(tmp, ctx->rows_total, ctx->B, ctx->Bp, ctx->opt.table_is_neglog,
                               (R*)ctx->table, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  cudaFree(tmp);
  if (ctx->precision == 32 && ctx->opt.table_texture != 2) {
    // the FP32 table also as a 1-D linear texture of float2 entries
    const size_t entries = (size_t)ctx->rows_total * ctx->Bp;
    cudaResourceDesc rd;
    memset(&rd, 0, sizeof(rd));
    rd.resType = cudaResourceTypeLinear;
    rd.res.linear.devPtr = ctx->table;
    rd.res.linear.desc = cudaCreateChannelDesc<float2>();
    rd.res.linear.sizeInBytes = entries * sizeof(float2);
    cudaTextureDesc td;
    memset(&td, 0, sizeof(td));
    td.readMode = cudaReadModeElementType;
    int maxw = 0;
    CK(ctx, cudaDeviceGetAttribute(&maxw, cudaDevAttrMaxTexture1DLinearWidth, ctx->device));
    if (entries <= (size_t)maxw && entries < (1ull << 31))
      CK(ctx, cudaCreateTextureObject(&ctx->tex, &rd, &td, nullptr));
    else if (ctx->opt.table_texture == 1)
      return set_err(ctx, AMH_EINVAL, "the table exceeds the 1-D texture limit");
  }
  // state
  const size_t tb = sizeof(R) * (size_t)ctx->tors_total;
  CK(ctx, cudaMalloc(&ctx->theta, tb));
  CK(ctx, cudaMalloc(&ctx->best_theta, tb));
  CK(ctx, cudaMalloc(&ctx->f32buf, sizeof(float) * (size_t)ctx->tors_total));
  CK(ctx, cudaMemcpy(ctx->f32buf, torsions, sizeof(float) * (size_t)ctx->tors_total,
                     cudaMemcpyHostToDevice));
  CK(ctx, launch_convert_in<R>(ctx->f32buf, (R*)ctx->theta, ctx->tors_total, ctx->stream));
  // kernels may use all of the opt-in shared memory
  for (int C = 1; C <= max_C(ctx->precision); C *= 2) CK(ctx, gset<R>(C, ctx->smem_optin));
  if (ctx->precision == 32) CK(ctx, gwarp_set_smem(ctx->smem_optin));
  if (ctx->opt.global_kernel == 2 && !warp_applies(ctx))
    return set_err(ctx, AMH_EINVAL, "the warp-per-chain kernel needs L <= 768");
  CK(ctx, local_set_smem<R>(ctx->smem_optin));
  CK(ctx, grad_set_smem<R>(ctx->smem_optin));
  // launch shape
  amh_status st;
  if (ctx->opt.chains_per_cta == 0) {
    st = autotune<R>(ctx);
  } else if (ctx->opt.global_kernel == 2) {
    st = configure_warp(ctx, ctx->opt.chains_per_cta,
                        ctx->opt.warps_per_chain ? ctx->opt.warps_per_chain : 1);
    if (st) return st;
    ctx->use_warp = true;
    st = configure_global<R>(ctx, 1, 128, 0);  // the energy kernel's shape
  } else {
    const int C = ctx->opt.chains_per_cta;
    const int T = ctx->opt.threads_per_cta ? ctx->opt.threads_per_cta : 256;
    // staged rows run every straddle pair: with the far-field skip on, a
    // fixed shape stages only when asked to
    const bool skip = ctx->precision == 32 && ctx->opt.far_pairs == 0 &&
                      ctx->Lmax <= kMaxChunks * kPairChunk + 1;
    const int D = ctx->opt.stage_table == 2 || (ctx->opt.stage_table == 0 && skip)
                      ? 0
                      : stage_depth_for(ctx, C, T);
    if (ctx->opt.stage_table == 1 && D == 0)
      return set_err(ctx, AMH_EINVAL, "table staging needs FP32, 4 or 8 chains per CTA and room");
    st = configure_global<R>(ctx, C, T, D);
  }
  if (st) return st;
  // local groups for every chains-per-CTA option
  for (int q = 0; q < 6; ++q) {
    st = upload_groups(ctx, make_groups(ctx, 1 << q), &ctx->lgroups_d[q], &ctx->nlgroups[q]);
    if (st) return st;
  }
  st = run_energy<R>(ctx);
  if (st) return st;
  st = run_best<R>(ctx, 1);
  if (st) return st;
  return check_err_flag(ctx);
}

// Most chains per CTA of a local sweep.
constexpr int kLocalMaxChains = 32;

template <class R>
amh_status sweep_impl(amh_ctx* ctx, int mode, int window, double T, double sigma, long long steps,
                      int are_sweeps, unsigned long long seed, int nsched = 0,
                      const double* Ts = nullptr, const double* Ss = nullptr) {
  SweepArgs<R> a = make_args<R>(ctx);
  a.T = T;
  a.sigma = (R)sigma;
  a.nsched = nsched;
  for (int q = 0; q < nsched; ++q) {
    a.sched_T[q] = Ts[q];
    a.sched_sigma[q] = (R)Ss[q];
  }
  a.seed = seed;
  a.steps = steps;
  a.steps_are_sweeps = are_sweeps;
  a.window = window;
  CK(ctx, cudaMemsetAsync(ctx->queue, 0, sizeof(int), ctx->stream));
  if (mode == AMH_GLOBAL) {
    if constexpr (sizeof(R) == 4) {
      if (ctx->use_warp) {
        a.groups = ctx->wgroups_d;
        a.ngroups = ctx->nwgroups;
        CK(ctx, launch_gwarp(a, ctx->warpW, ctx->warpG, ctx->grid_warp, ctx->stream));
        return AMH_OK;
      }
    }
    CK(ctx, glaunch<R>(false, ctx->C, ctx->stage_depth > 0, a, ctx->threads, ctx->grid_global,
                       ctx->stream));
  } else {
    const int h = window / 2;
    const int ncol = std::max(4 * h, 1);
    const int cnt = (ctx->nmax + ncol - 1) / ncol;
    int q = 0;
    while (q < 5 && (2 << q) <= kLocalMaxChains && (2 << q) * cnt <= 256) ++q;
    // 256 threads (measured faster than one thread per window of a colour:
    // the idle lanes cost less than the extra CTAs); fewer chains per CTA,
    // then fewer threads, until shared memory fits
    const size_t room = ctx->smem_optin - kStaticSmemMargin;
    int threads = 256;
    size_t sm = 0;
    if (ctx->opt.local_chains_per_cta || ctx->opt.local_threads) {
      // a given shape
      q = 0;
      if (ctx->opt.local_chains_per_cta)
        while ((1 << q) < ctx->opt.local_chains_per_cta) ++q;
      threads = ctx->opt.local_threads ? ctx->opt.local_threads : 256;
      sm = local_smem_bytes<R>(ctx->nmax, 1 << q, threads, window);
      if (sm > room) return set_err(ctx, AMH_EINVAL, "local launch shape does not fit shared memory");
    }
    for (; q >= 0 && !ctx->opt.local_chains_per_cta && !ctx->opt.local_threads; --q) {
      threads = 256;
      for (;;) {
        sm = local_smem_bytes<R>(ctx->nmax, 1 << q, threads, window);
        if (sm <= room || threads == 32) break;
        threads = std::max(32, (threads / 2 + 31) / 32 * 32);
      }
      if (sm <= room) break;
    }
    if (q < 0 || sm > room) return set_err(ctx, AMH_EINVAL, "window too large for shared memory");
    const int Gc = 1 << q;
    a.groups = ctx->lgroups_d[q];
    a.ngroups = ctx->nlgroups[q];
    const int per_sm = std::max(1, std::min((int)(ctx->smem_optin / std::max<size_t>(sm, 1)),
                                            2048 / threads));
    const int grid = std::max(1, std::min(a.ngroups, ctx->sm_count * per_sm));
    CK(ctx, launch_local<R>(a, Gc, threads, grid, ctx->stream));
  }
  return AMH_OK;
}

amh_status check_ctx(amh_ctx* ctx) {
  if (!ctx) return AMH_ESTATE;
  if (ctx->broken) return AMH_ESTATE;
  cudaError_t e = cudaSetDevice(ctx->device);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "cudaSetDevice");
  return AMH_OK;
}

void free_ctx(amh_ctx* ctx) {
  if (!ctx) return;
  cudaSetDevice(ctx->device);
  if (ctx->stream) cudaStreamSynchronize(ctx->stream);
  if (ctx->tex) cudaDestroyTextureObject(ctx->tex);
  void* ptrs[] = {ctx->table, ctx->theta, ctx->best_theta, ctx->f32buf, ctx->tcount, ctx->E_cur,
                  ctx->best_E, ctx->acc, ctx->prot_d, ctx->chain_prot_d, ctx->ggroups_d,
                  ctx->queue, ctx->err, ctx->trace, ctx->trace_count, ctx->ladder,
                  ctx->pair_count, ctx->coords, ctx->wgroups_d, ctx->tcache};
  for (void* p : ptrs)
    if (p) cudaFree(p);
  for (int q = 0; q < 6; ++q)
    if (ctx->lgroups_d[q]) cudaFree(ctx->lgroups_d[q]);
  delete ctx;
}

}  // namespace

namespace amh {
void set_context_free_error(const std::string& m) { g_free_error = m; }
}  // namespace amh

extern "C" {

void amh_options_default(amh_options* opt) {
  if (!opt) return;
  memset(opt, 0, sizeof(*opt));
  opt->precision = 32;
  opt->resync_every = 1000;
  opt->chains_per_cta = 0;
  opt->threads_per_cta = 0;
  opt->trace_chains = 0;
  opt->trace_capacity = 0;
  opt->lattice_K = 0;
  opt->table_is_neglog = 0;
  opt->stage_table = 0;
  opt->table_texture = 0;
  opt->far_pairs = 0;
  opt->local_chains_per_cta = 0;
  opt->local_threads = 0;
  opt->stream = nullptr;
  opt->keep_coords = 0;
  opt->wait_test = 0;
  opt->global_kernel = 0;
  opt->warps_per_chain = 0;
}

amh_status amh_init(amh_ctx** out, int n_proteins, const int* L, const int* chains_per_protein,
                    const float* torsions, const double* table, const double* edges, int B,
                    const amh_options* opt) {
  if (!out) return set_err(nullptr, AMH_EINVAL, "out is NULL");
  *out = nullptr;
  if (n_proteins < 1 || !L || !chains_per_protein || !torsions || !table || !edges)
    return set_err(nullptr, AMH_EINVAL, "missing argument");
  if (B < 2 || B > 256) return set_err(nullptr, AMH_EINVAL, "B must be in [2, 256]");
  amh_options o;
  if (opt)
    o = *opt;
  else
    amh_options_default(&o);
  if (o.precision != 32 && o.precision != 64)
    return set_err(nullptr, AMH_EINVAL, "precision must be 32 or 64");
  if (o.resync_every <= 0) o.resync_every = 1000;
  if (o.chains_per_cta != 0 && o.chains_per_cta != 1 && o.chains_per_cta != 2 &&
      o.chains_per_cta != 4 && o.chains_per_cta != 8)
    return set_err(nullptr, AMH_EINVAL, "chains_per_cta must be 0, 1, 2, 4 or 8");
  if (o.precision == 64 && o.chains_per_cta == 8)
    return set_err(nullptr, AMH_EINVAL, "precision 64 allows at most 4 chains per CTA");
  if (o.threads_per_cta != 0 && o.threads_per_cta != 64 && o.threads_per_cta != 128 &&
      o.threads_per_cta != 256 && o.threads_per_cta != 512)
    return set_err(nullptr, AMH_EINVAL, "threads_per_cta must be 0, 64, 128, 256 or 512");
  if (o.table_texture < 0 || o.table_texture > 2)
    return set_err(nullptr, AMH_EINVAL, "table_texture must be 0, 1 or 2");
  if (o.stage_table < 0 || o.stage_table > 2)
    return set_err(nullptr, AMH_EINVAL, "stage_table must be 0, 1 or 2");
  if (o.far_pairs < 0 || o.far_pairs > 1)
    return set_err(nullptr, AMH_EINVAL, "far_pairs must be 0 or 1");
  if (o.local_chains_per_cta < 0 || o.local_chains_per_cta > kLocalMaxChains ||
      (o.local_chains_per_cta & (o.local_chains_per_cta - 1)))
    return set_err(nullptr, AMH_EINVAL, "local_chains_per_cta must be 0, 1, 2, 4, 8, 16 or 32");
  if (o.local_threads < 0 || o.local_threads > 256 || o.local_threads % 32)
    return set_err(nullptr, AMH_EINVAL, "local_threads must be 0 or a multiple of 32 up to 256");
  if (o.trace_chains < 0 || o.trace_capacity < 0 || o.lattice_K < 0)
    return set_err(nullptr, AMH_EINVAL, "negative option");
  if (o.keep_coords < 0 || o.keep_coords > 1)
    return set_err(nullptr, AMH_EINVAL, "keep_coords must be 0 or 1");
  if (o.wait_test < 0) return set_err(nullptr, AMH_EINVAL, "wait_test must be >= 0");
  if (o.global_kernel < 0 || o.global_kernel > 2)
    return set_err(nullptr, AMH_EINVAL, "global_kernel must be 0, 1 or 2");
  if (o.warps_per_chain != 0 && o.warps_per_chain != 1 && o.warps_per_chain != 2 &&
      o.warps_per_chain != 4)
    return set_err(nullptr, AMH_EINVAL, "warps_per_chain must be 0, 1, 2 or 4");
  if (o.global_kernel == 2 && o.chains_per_cta * (o.warps_per_chain ? o.warps_per_chain : 1) > 8)
    return set_err(nullptr, AMH_EINVAL, "at most 8 warps per CTA");
  if (o.global_kernel == 2 &&
      (o.precision != 32 || o.far_pairs != 0 || o.stage_table == 1 || o.threads_per_cta != 0))
    return set_err(nullptr, AMH_EINVAL,
                   "the warp-per-chain kernel needs precision 32, far_pairs 0, no staging and no "
                   "threads_per_cta");
  // bins: evenly spaced centres
  for (int j = 0; j < B; ++j)
    if (!(edges[j] < edges[j + 1]) || !std::isfinite(edges[j]))
      return set_err(nullptr, AMH_EINVAL, "edges must be finite and ascending (last may be +inf)");
  std::vector<double> cen(B);
  for (int j = 0; j < B; ++j) {
    if (std::isinf(edges[j + 1])) {
      if (j == 0) return set_err(nullptr, AMH_EINVAL, "open first bin");
      cen[j] = edges[j] + 0.5 * (edges[j] - edges[j - 1]);
    } else {
      cen[j] = 0.5 * (edges[j] + edges[j + 1]);
    }
  }
  const double w = (cen[B - 1] - cen[0]) / (B - 1);
  for (int j = 0; j + 1 < B; ++j)
    if (std::fabs((cen[j + 1] - cen[j]) - w) > 1e-9 * w)
      return set_err(nullptr, AMH_EINVAL, "bin centres are not evenly spaced");

  amh_ctx* ctx = new amh_ctx();
  ctx->opt = o;
  ctx->precision = o.precision;
  ctx->stream = (cudaStream_t)o.stream;
  ctx->B = B;
  ctx->Bp = (B + 1) & ~1;  // (value, slope) entries per row: even, so rows are 16-byte aligned
  ctx->c0 = cen[0];
  ctx->w = w;
  ctx->nprot = n_proteins;
  long long chain0 = 0, tors0 = 0, rows = 0;
  for (int p = 0; p < n_proteins; ++p) {
    if (L[p] < 2 || L[p] > 4096 || chains_per_protein[p] < 1) {
      delete ctx;
      return set_err(nullptr, AMH_EINVAL, "need 2 <= L <= 4096 and >= 1 chain per protein");
    }
    ProteinDev d;
    d.L = L[p];
    d.n = 2 * L[p];
    d.tab_off = rows * ctx->Bp;
    d.chain0 = (int)chain0;
    d.nchains = chains_per_protein[p];
    d.tors0 = tors0;
    ctx->prot_h.push_back(d);
    ctx->L.push_back(L[p]);
    ctx->nch.push_back(chains_per_protein[p]);
    ctx->t_host.push_back(0);
    chain0 += chains_per_protein[p];
    tors0 += (long long)chains_per_protein[p] * d.n;
    rows += (long long)L[p] * (L[p] - 1) / 2;
    ctx->Lmax = std::max(ctx->Lmax, L[p]);
  }
  if (chain0 > (1LL << 30)) {
    delete ctx;
    return set_err(nullptr, AMH_EINVAL, "too many chains");
  }
  ctx->nmax = 2 * ctx->Lmax;
  ctx->total_chains = (int)chain0;
  ctx->tors_total = tors0;
  ctx->rows_total = rows;

  cudaError_t e = cudaGetDevice(&ctx->device);
  if (e != cudaSuccess) {
    delete ctx;
    return set_err(nullptr, AMH_ECUDA, std::string("no CUDA device: ") + cudaGetErrorString(e));
  }
  cudaDeviceProp prop;
  e = cudaGetDeviceProperties(&prop, ctx->device);
  if (e != cudaSuccess) {
    delete ctx;
    return set_err(nullptr, AMH_ECUDA, cudaGetErrorString(e));
  }
  ctx->sm_count = prop.multiProcessorCount;
  ctx->smem_optin = prop.sharedMemPerBlockOptin;

  auto bail = [&](amh_status st) {
    g_free_error = ctx->msg;
    free_ctx(ctx);
    return st;
  };
#define CKI(call)                                                        \
  do {                                                                   \
    cudaError_t e_ = (call);                                             \
    if (e_ != cudaSuccess) return bail(cuda_fail(ctx, e_, #call));       \
  } while (0)
  const int nc = ctx->total_chains;
  CKI(cudaMalloc(&ctx->tcount, sizeof(long long) * nc));
  CKI(cudaMemset(ctx->tcount, 0, sizeof(long long) * nc));
  CKI(cudaMalloc(&ctx->E_cur, sizeof(double) * nc));
  CKI(cudaMalloc(&ctx->best_E, sizeof(double) * nc));
  CKI(cudaMalloc(&ctx->acc, sizeof(long long) * nc));
  CKI(cudaMemset(ctx->acc, 0, sizeof(long long) * nc));
  CKI(cudaMalloc(&ctx->prot_d, sizeof(ProteinDev) * n_proteins));
  CKI(cudaMemcpy(ctx->prot_d, ctx->prot_h.data(), sizeof(ProteinDev) * n_proteins,
                 cudaMemcpyHostToDevice));
  std::vector<int> cp(nc);
  for (int p = 0; p < n_proteins; ++p)
    for (int c = 0; c < ctx->nch[p]; ++c) cp[ctx->prot_h[p].chain0 + c] = p;
  CKI(cudaMalloc(&ctx->chain_prot_d, sizeof(int) * nc));
  CKI(cudaMemcpy(ctx->chain_prot_d, cp.data(), sizeof(int) * nc, cudaMemcpyHostToDevice));
  CKI(cudaMalloc(&ctx->queue, sizeof(int)));
  CKI(cudaMalloc(&ctx->err, sizeof(int)));
  CKI(cudaMemset(ctx->err, 0, sizeof(int)));
  CKI(cudaMalloc(&ctx->pair_count, 2 * sizeof(unsigned long long)));
  CKI(cudaMemset(ctx->pair_count, 0, 2 * sizeof(unsigned long long)));
  if (o.keep_coords) {
    // 3 values per residue per chain: half the torsion count times 3
    const size_t rs = o.precision == 64 ? sizeof(double) : sizeof(float);
    CKI(cudaMalloc(&ctx->coords, rs * 3 * (size_t)(ctx->tors_total / 2)));
  }
  if (o.trace_chains > 0 && o.trace_capacity > 0) {
    const int tc = std::min(o.trace_chains, nc);
    ctx->opt.trace_chains = tc;
    CKI(cudaMalloc(&ctx->trace, sizeof(TraceRec) * (size_t)tc * o.trace_capacity));
    CKI(cudaMalloc(&ctx->trace_count, sizeof(long long) * tc));
    CKI(cudaMemset(ctx->trace_count, 0, sizeof(long long) * tc));
  } else {
    ctx->opt.trace_chains = 0;
  }
  // the memsets above ran on the legacy stream; a non-blocking context
  // stream is not ordered after it
  CKI(cudaDeviceSynchronize());
#undef CKI
  amh_status st = ctx->precision == 64 ? init_impl<double>(ctx, torsions, table)
                                       : init_impl<float>(ctx, torsions, table);
  if (st != AMH_OK) return bail(st);
  *out = ctx;
  return AMH_OK;
}

// Recompute E_cur if the state was replaced since it was last computed.
static amh_status fresh_energy(amh_ctx* ctx) {
  if (!ctx->energy_stale) return AMH_OK;
  amh_status st = ctx->precision == 64 ? run_energy<double>(ctx) : run_energy<float>(ctx);
  if (st) return st;
  ctx->energy_stale = false;
  return AMH_OK;
}

amh_status amh_energy(amh_ctx* ctx, double* E_out) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  st = ctx->precision == 64 ? run_energy<double>(ctx) : run_energy<float>(ctx);
  if (st) return st;
  ctx->energy_stale = false;
  if (E_out) {
    CK(ctx, cudaMemcpyAsync(E_out, ctx->E_cur, sizeof(double) * ctx->total_chains,
                            cudaMemcpyDefault, ctx->stream));
    if (!is_device_ptr(E_out)) return check_err_flag(ctx);
  }
  return AMH_OK;
}

static amh_status sweep_common(amh_ctx* ctx, int mode, int window, double T, double sigma,
                               long long steps, int are_sweeps, unsigned long long seed,
                               long long* accepted_out, int nsched = 0,
                               const double* Ts = nullptr, const double* Ss = nullptr) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  if (mode != AMH_LOCAL && mode != AMH_GLOBAL) return set_err(ctx, AMH_EINVAL, "bad mode");
  if (!(T > 0) || !std::isfinite(T)) return set_err(ctx, AMH_EINVAL, "T must be positive");
  if (!std::isfinite(sigma)) return set_err(ctx, AMH_EINVAL, "sigma must be finite");
  if (steps < 0) return set_err(ctx, AMH_EINVAL, "steps must be >= 0");
  for (int q = 0; q < nsched; ++q) {
    if (!(Ts[q] > 0) || !std::isfinite(Ts[q]))
      return set_err(ctx, AMH_EINVAL, "every T[q] must be positive");
    if (!std::isfinite(Ss[q])) return set_err(ctx, AMH_EINVAL, "every sigma[q] must be finite");
  }
  if (nsched)
    for (int p = 0; p < ctx->nprot; ++p)
      if (ctx->t_host[p] % (2LL * ctx->L[p]) != 0)
        return set_err(ctx, AMH_EINVAL, "a scheduled run starts on a sweep boundary");
  if (mode == AMH_LOCAL) {
    if (window < 0 || window > 64) return set_err(ctx, AMH_EINVAL, "window must be in [0, 64]");
    for (int p = 0; p < ctx->nprot; ++p) {
      const long long n = 2LL * ctx->L[p];
      if (ctx->t_host[p] % n != 0 || (!are_sweeps && steps % n != 0))
        return set_err(ctx, AMH_EINVAL, "local sweeps need whole sweeps (t and steps multiples of n)");
    }
  }
  if (steps > 0) {
    st = ctx->precision == 64
             ? sweep_impl<double>(ctx, mode, window, T, sigma, steps, are_sweeps, seed, nsched,
                                  Ts, Ss)
             : sweep_impl<float>(ctx, mode, window, T, sigma, steps, are_sweeps, seed, nsched,
                                 Ts, Ss);
    if (st) return st;
    if (mode == AMH_GLOBAL) ctx->energy_stale = false;  // every chain ends with V from scratch
  } else {
    CK(ctx, cudaMemsetAsync(ctx->acc, 0, sizeof(long long) * ctx->total_chains, ctx->stream));
  }
  for (int p = 0; p < ctx->nprot; ++p)
    ctx->t_host[p] += are_sweeps ? steps * 2LL * ctx->L[p] : steps;
  if (accepted_out) {
    CK(ctx, cudaMemcpyAsync(accepted_out, ctx->acc, sizeof(long long) * ctx->total_chains,
                            cudaMemcpyDefault, ctx->stream));
    if (!is_device_ptr(accepted_out)) return check_err_flag(ctx);
  }
  return AMH_OK;
}

amh_status amh_sweep(amh_ctx* ctx, int mode, int window, double T, double sigma_rad,
                     long long steps, unsigned long long seed, long long* accepted_out) {
  return sweep_common(ctx, mode, window, T, sigma_rad, steps, 0, seed, accepted_out);
}

amh_status amh_sweeps(amh_ctx* ctx, int mode, int window, double T, double sigma_rad,
                      long long nsweeps, unsigned long long seed, long long* accepted_out) {
  return sweep_common(ctx, mode, window, T, sigma_rad, nsweeps, 1, seed, accepted_out);
}

amh_status amh_sweeps_sched(amh_ctx* ctx, int mode, int window, int nsweeps, const double* T,
                            const double* sigma_rad, unsigned long long seed,
                            long long* accepted_out) {
  if (ctx && (nsweeps < 1 || nsweeps > AMH_MAX_SCHED || !T || !sigma_rad))
    return set_err(ctx, AMH_EINVAL, "need 1 <= nsweeps <= AMH_MAX_SCHED and T, sigma arrays");
  return sweep_common(ctx, mode, window, ctx ? T[0] : 1.0, ctx ? sigma_rad[0] : 0.0, nsweeps, 1,
                      seed, accepted_out, nsweeps, T, sigma_rad);
}

amh_status amh_grad(amh_ctx* ctx, int protein, const void* theta, int batch, double* E_out,
                    void* dE_dtheta) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  if (protein < 0 || protein >= ctx->nprot || batch < 0)
    return set_err(ctx, AMH_EINVAL, "bad protein or batch");
  if (batch == 0) return AMH_OK;
  if (!is_device_ptr(theta) || !is_device_ptr(E_out) || !is_device_ptr(dE_dtheta))
    return set_err(ctx, AMH_EINVAL, "amh_grad needs device pointers");
  const int L = ctx->L[protein];
  const size_t esz = ctx->precision == 64 ? 8 : 4;
  const size_t sm = grad_smem_bytes(esz, L);
  if (sm > ctx->smem_optin - kStaticSmemMargin)
    return set_err(ctx, AMH_EINVAL, "protein too long for amh_grad");
  if (ctx->precision == 64) {
    CK(ctx, launch_grad<double>(&ctx->prot_h[protein], protein, L, (const double*)theta, batch,
                                E_out, (double*)dE_dtheta, make_tab<double>(ctx),
                                ideal_geometry<double>(), ctx->stream));
  } else {
    CK(ctx, launch_grad<float>(&ctx->prot_h[protein], protein, L, (const float*)theta, batch,
                               E_out, (float*)dE_dtheta, make_tab<float>(ctx),
                               ideal_geometry<float>(), ctx->stream));
  }
  return AMH_OK;
}

amh_status amh_get_state(amh_ctx* ctx, float* torsions_out, double* E_out, double* best_E,
                         float* best_torsions) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  bool host = false;
  const long long nt = ctx->tors_total;
  auto out_tors = [&](const void* src, float* dst) -> amh_status {
    if (!dst) return AMH_OK;
    if (ctx->precision == 64) {
      CK(ctx, launch_convert_out<double>((const double*)src, ctx->f32buf, nt, ctx->stream));
      CK(ctx, cudaMemcpyAsync(dst, ctx->f32buf, sizeof(float) * nt, cudaMemcpyDefault, ctx->stream));
    } else {
      CK(ctx, cudaMemcpyAsync(dst, src, sizeof(float) * nt, cudaMemcpyDefault, ctx->stream));
    }
    if (!is_device_ptr(dst)) host = true;
    if (ctx->precision == 64) CK(ctx, cudaStreamSynchronize(ctx->stream));
    return AMH_OK;
  };
  st = out_tors(ctx->theta, torsions_out);
  if (st) return st;
  st = out_tors(ctx->best_theta, best_torsions);
  if (st) return st;
  if (E_out) {
    st = fresh_energy(ctx);
    if (st) return st;
    CK(ctx, cudaMemcpyAsync(E_out, ctx->E_cur, sizeof(double) * ctx->total_chains,
                            cudaMemcpyDefault, ctx->stream));
    if (!is_device_ptr(E_out)) host = true;
  }
  if (best_E) {
    CK(ctx, cudaMemcpyAsync(best_E, ctx->best_E, sizeof(double) * ctx->total_chains,
                            cudaMemcpyDefault, ctx->stream));
    if (!is_device_ptr(best_E)) host = true;
  }
  if (host) CK(ctx, cudaStreamSynchronize(ctx->stream));
  return AMH_OK;
}

amh_status amh_set_state(amh_ctx* ctx, const float* torsions) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  if (!torsions) return set_err(ctx, AMH_EINVAL, "torsions is NULL");
  const long long nt = ctx->tors_total;
  if (ctx->precision == 64) {
    CK(ctx, cudaMemcpyAsync(ctx->f32buf, torsions, sizeof(float) * nt, cudaMemcpyDefault,
                            ctx->stream));
    CK(ctx, launch_convert_in<double>(ctx->f32buf, (double*)ctx->theta, nt, ctx->stream));
  } else {
    // the FP32 form holds the torsions as given: one copy, no conversion
    CK(ctx, cudaMemcpyAsync(ctx->theta, torsions, sizeof(float) * nt, cudaMemcpyDefault,
                            ctx->stream));
  }
  ctx->energy_stale = true;  // V is recomputed when next read, unless a global sweep does it
  if (!is_device_ptr(torsions)) CK(ctx, cudaStreamSynchronize(ctx->stream));
  return AMH_OK;
}

amh_status amh_noisy_restart(amh_ctx* ctx, double sd_rad, unsigned long long seed) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  if (!std::isfinite(sd_rad) || sd_rad < 0) return set_err(ctx, AMH_EINVAL, "bad sd");
  if (ctx->precision == 64)
    CK(ctx, launch_noisy<double>(ctx->prot_d, ctx->chain_prot_d, ctx->total_chains, ctx->nmax,
                                 (double*)ctx->theta, sd_rad, seed, ctx->stream));
  else
    CK(ctx, launch_noisy<float>(ctx->prot_d, ctx->chain_prot_d, ctx->total_chains, ctx->nmax,
                                (float*)ctx->theta, (float)sd_rad, seed, ctx->stream));
  ctx->energy_stale = true;  // V is recomputed when next read, unless a global sweep does it
  return AMH_OK;
}

amh_status amh_get_trace(amh_ctx* ctx, int chain, amh_trace_rec* out, long long* count) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  if (!ctx->trace || chain < 0 || chain >= ctx->opt.trace_chains)
    return set_err(ctx, AMH_EINVAL, "chain is not traced");
  long long cnt = 0;
  CK(ctx, cudaMemcpyAsync(&cnt, ctx->trace_count + chain, sizeof(long long),
                          cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  if (count) *count = cnt;
  if (out && cnt > 0) {
    static_assert(sizeof(amh_trace_rec) == sizeof(TraceRec), "trace record layout");
    CK(ctx, cudaMemcpyAsync(out, ctx->trace + (size_t)chain * ctx->opt.trace_capacity,
                            sizeof(TraceRec) * (size_t)cnt, cudaMemcpyDefault, ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return AMH_OK;
}

amh_status amh_set_ladder(amh_ctx* ctx, int K, const double* ladder) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  if (K == 0) {
    ctx->ladder_K = 0;
    return AMH_OK;
  }
  if (K < 2 || !ladder) return set_err(ctx, AMH_EINVAL, "a ladder needs K >= 2 factors");
  for (int p = 0; p < ctx->nprot; ++p)
    if (ctx->nch[p] % K != 0)
      return set_err(ctx, AMH_EINVAL, "every protein's chain count must be a multiple of K");
  for (int j = 0; j < K; ++j)
    if (!(ladder[j] > 0) || !std::isfinite(ladder[j]))
      return set_err(ctx, AMH_EINVAL, "ladder factors must be positive");
  if (ctx->ladder) {
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    cudaFree(ctx->ladder);
    ctx->ladder = nullptr;
  }
  CK(ctx, cudaMalloc(&ctx->ladder, sizeof(double) * K));
  CK(ctx, cudaMemcpy(ctx->ladder, ladder, sizeof(double) * K, cudaMemcpyHostToDevice));
  ctx->ladder_K = K;
  return AMH_OK;
}

amh_status amh_exchange(amh_ctx* ctx, double T, int parity, unsigned long long seed,
                        long long* swapped_out) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  if (!ctx->ladder_K) return set_err(ctx, AMH_EINVAL, "no temperature ladder set");
  if (!(T > 0) || !std::isfinite(T) || (parity != 0 && parity != 1))
    return set_err(ctx, AMH_EINVAL, "T must be positive and parity 0 or 1");
  st = fresh_energy(ctx);
  if (st) return st;
  if (ctx->precision == 64) {
    CK(ctx, launch_exchange<double>(ctx->prot_d, ctx->chain_prot_d, ctx->total_chains,
                                    ctx->ladder_K, ctx->ladder, T, parity, seed, ctx->xround,
                                    (double*)ctx->theta, ctx->E_cur, ctx->acc, ctx->stream));
  } else {
    CK(ctx, launch_exchange<float>(ctx->prot_d, ctx->chain_prot_d, ctx->total_chains,
                                   ctx->ladder_K, ctx->ladder, T, parity, seed, ctx->xround,
                                   (float*)ctx->theta, ctx->E_cur, ctx->acc, ctx->stream));
  }
  ++ctx->xround;
  if (swapped_out) {
    CK(ctx, cudaMemcpyAsync(swapped_out, ctx->acc, sizeof(long long) * ctx->total_chains,
                            cudaMemcpyDefault, ctx->stream));
    if (!is_device_ptr(swapped_out)) CK(ctx, cudaStreamSynchronize(ctx->stream));
  }
  return AMH_OK;
}

amh_status amh_counter(amh_ctx* ctx, int chain, long long* t) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  if (chain < 0 || chain >= ctx->total_chains || !t) return set_err(ctx, AMH_EINVAL, "bad chain");
  CK(ctx, cudaMemcpyAsync(t, ctx->tcount + chain, sizeof(long long), cudaMemcpyDeviceToHost,
                          ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  return AMH_OK;
}

amh_status amh_pair_terms(amh_ctx* ctx, unsigned long long* evaluated,
                          unsigned long long* formed) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  if (!evaluated) return set_err(ctx, AMH_EINVAL, "evaluated is NULL");
  unsigned long long v[2];
  CK(ctx, cudaMemcpyAsync(v, ctx->pair_count, sizeof(v), cudaMemcpyDeviceToHost, ctx->stream));
  CK(ctx, cudaStreamSynchronize(ctx->stream));
  *evaluated = v[1];
  if (formed) *formed = v[0];
  return AMH_OK;
}

amh_status amh_philox(unsigned long long seed, unsigned chain, unsigned long long t0,
                      unsigned stream, long long count, unsigned* words_out, float* z_out,
                      float* u_out) {
  if (count < 0) return set_err(nullptr, AMH_EINVAL, "count < 0");
  if (count == 0) return AMH_OK;
  uint4* w = nullptr;
  float *z = nullptr, *u = nullptr;
  auto fail = [&](cudaError_t e, const char* what) {
    if (w) cudaFree(w);
    if (z) cudaFree(z);
    if (u) cudaFree(u);
    return set_err(nullptr, AMH_ECUDA, std::string(what) + ": " + cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = cudaMalloc(&w, sizeof(uint4) * count)) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&z, sizeof(float) * count)) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = cudaMalloc(&u, sizeof(float) * count)) != cudaSuccess) return fail(e, "cudaMalloc");
  if ((e = launch_philox_fill(seed, chain, t0, stream, count, w, z, u, 0)) != cudaSuccess)
    return fail(e, "philox kernel");
  if (words_out && (e = cudaMemcpy(words_out, w, sizeof(uint4) * count, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return fail(e, "cudaMemcpy");
  if (z_out && (e = cudaMemcpy(z_out, z, sizeof(float) * count, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return fail(e, "cudaMemcpy");
  if (u_out && (e = cudaMemcpy(u_out, u, sizeof(float) * count, cudaMemcpyDeviceToHost)) != cudaSuccess)
    return fail(e, "cudaMemcpy");
  cudaFree(w);
  cudaFree(z);
  cudaFree(u);
  return AMH_OK;
}

amh_status amh_get_coords(amh_ctx* ctx, double* cb_out) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  if (!ctx->coords) return set_err(ctx, AMH_EINVAL, "coordinates are kept only with keep_coords = 1");
  if (!cb_out) return set_err(ctx, AMH_EINVAL, "cb_out is NULL");
  st = fresh_energy(ctx);  // a replaced state: G(s) and V are rebuilt together
  if (st) return st;
  const size_t cnt = 3 * (size_t)(ctx->tors_total / 2);
  if (ctx->precision == 64) {
    CK(ctx, cudaMemcpyAsync(cb_out, ctx->coords, sizeof(double) * cnt, cudaMemcpyDeviceToHost,
                            ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
  } else {
    std::vector<float> h(cnt);
    CK(ctx, cudaMemcpyAsync(h.data(), ctx->coords, sizeof(float) * cnt, cudaMemcpyDeviceToHost,
                            ctx->stream));
    CK(ctx, cudaStreamSynchronize(ctx->stream));
    for (size_t i = 0; i < cnt; ++i) cb_out[i] = (double)h[i];
  }
  return check_err_flag(ctx);
}

amh_status amh_window_coords(amh_ctx* ctx, int chain, int k, int window, double* cb_out,
                             int* lo_out, int* hi_out) {
  amh_status st = check_ctx(ctx);
  if (st) return st;
  if (chain < 0 || chain >= ctx->total_chains) return set_err(ctx, AMH_EINVAL, "bad chain");
  if (window < 0 || window > 64) return set_err(ctx, AMH_EINVAL, "window must be in [0, 64]");
  if (!cb_out) return set_err(ctx, AMH_EINVAL, "cb_out is NULL");
  int p = 0;
  while (p + 1 < ctx->nprot && chain >= ctx->prot_h[p + 1].chain0) ++p;
  const ProteinDev& P = ctx->prot_h[p];
  if (k < 0 || k >= P.n) return set_err(ctx, AMH_EINVAL, "k must be in [0, 2L)");
  const int h = window / 2, i = k >> 1;
  const int lo = std::max(0, i - h), hi = std::min(P.L - 1, i + h);
  const int cnt = 3 * (hi - lo + 1);
  const long long off = P.tors0 + (long long)(chain - P.chain0) * P.n;
  const size_t rs = ctx->precision == 64 ? sizeof(double) : sizeof(float);
  void* d = nullptr;
  CK(ctx, cudaMalloc(&d, rs * cnt));
  cudaError_t e;
  if (ctx->precision == 64)
    e = launch_window_coords<double>((const double*)ctx->theta + off, P.L, k, window,
                                     ideal_geometry<double>(), (double*)d, ctx->stream);
  else
    e = launch_window_coords<float>((const float*)ctx->theta + off, P.L, k, window,
                                    ideal_geometry<float>(), (float*)d, ctx->stream);
  std::vector<unsigned char> h_(rs * cnt);
  if (e == cudaSuccess) e = cudaMemcpyAsync(h_.data(), d, rs * cnt, cudaMemcpyDeviceToHost, ctx->stream);
  if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
  cudaFree(d);
  if (e != cudaSuccess) return cuda_fail(ctx, e, "window coordinates");
  for (int q = 0; q < cnt; ++q)
    cb_out[q] = ctx->precision == 64 ? ((const double*)h_.data())[q]
                                     : (double)((const float*)h_.data())[q];
  if (lo_out) *lo_out = lo;
  if (hi_out) *hi_out = hi;
  return AMH_OK;
}

const char* amh_last_error(const amh_ctx* ctx) {
  return ctx ? ctx->msg.c_str() : g_free_error.c_str();
}

amh_status amh_launch_config(amh_ctx* ctx, int* chains_per_cta, int* threads_per_cta,
                             int* stage_depth, int* kernel) {
  if (!ctx) return AMH_ESTATE;
  if (chains_per_cta) *chains_per_cta = ctx->use_warp ? ctx->warpW : ctx->C;
  if (threads_per_cta) *threads_per_cta = ctx->use_warp ? 32 * ctx->warpW * ctx->warpG : ctx->threads;
  if (stage_depth) *stage_depth = ctx->use_warp ? 0 : ctx->stage_depth;
  if (kernel) *kernel = ctx->use_warp ? 2 : 1;
  return AMH_OK;
}

void amh_destroy(amh_ctx* ctx) { free_ctx(ctx); }

}  // extern "C"
