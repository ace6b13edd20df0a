// amh_internal.h -- launch arguments and launchers shared by the library's
// translation units (not part of the public ABI).
#pragma once

#include <cmath>
#include <cstdint>
#include <string>
#include <cuda_runtime.h>

#include "amh.h"
#include "amh_device.cuh"

namespace amh {

// Ideal geometry of G(s) (bond lengths and angles listed in amh.h) as the
// (-b cos a, b sin a) pairs the builders use, computed in double precision.
template <class R>
inline Geom<R> ideal_geometry() {
  const double d2r = 3.14159265358979323846 / 180.0;
  const double bNCA = 1.458, bCAC = 1.525, bCN = 1.329, bCACB = 1.52;
  const double aNCAC = 111.2 * d2r, aCACN = 116.2 * d2r, aCNCA = 121.7 * d2r;
  const double aCCACB = 109.5 * d2r, tCB = 122.6 * d2r;
  Geom<R> g;
  g.bNCA = (R)bNCA;
  g.bCAC = (R)bCAC;
  g.cosNCAC = (R)std::cos(aNCAC);
  g.sinNCAC = (R)std::sin(aNCAC);
  g.pN_c = (R)(-bCN * std::cos(aCACN));
  g.pN_s = (R)(bCN * std::sin(aCACN));
  g.pCA_c = (R)(-bNCA * std::cos(aCNCA));
  g.pCA_s = (R)(bNCA * std::sin(aCNCA));
  g.pC_c = (R)(-bCAC * std::cos(aNCAC));
  g.pC_s = (R)(bCAC * std::sin(aNCAC));
  g.pCB_c = (R)(-bCACB * std::cos(aCCACB));
  g.pCB_s = (R)(bCACB * std::sin(aCCACB));
  g.cbT_c = (R)std::cos(tCB);
  g.cbT_s = (R)std::sin(tCB);
  return g;
}

// Message returned by amh_last_error(NULL) (calls without a context).
void set_context_free_error(const std::string& m);

// Arguments of a sweep / energy launch over chain groups.
// Fixed-side atoms per item of the global sweeps' pair loop, and per
// bounding sphere of the far-field test (one bit per chunk in a 64-bit word).
constexpr int kPairChunk = 12;
using ChunkBits = unsigned long long;
constexpr int kMaxChunks = 64;

// Sweeps of one scheduled call (amh_sweeps_sched) at most.
constexpr int kMaxSched = AMH_MAX_SCHED;

template <class R>
struct SweepArgs {
  const ProteinDev* prot;
  const GroupDev* groups;
  int ngroups;
  int* queue;  // work counter, zeroed before the launch
  R* theta;    // all chains' torsions (ragged, ProteinDev::tors0)
  R* best_theta;
  long long* tcount;  // per chain proposal counter
  double* E_cur;
  double* best_E;
  long long* acc_out;  // per chain accepted count of this call (may be null)
  Tab<R> tab;
  Geom<R> geom;
  Geom<double> geom64;  // the resync rebuilds G(s) in FP64 (stored in R)
  double T;
  R sigma;
  unsigned long long seed;
  long long steps;      // proposals per chain, or sweeps if steps_are_sweeps
  int steps_are_sweeps;
  int resync_every;
  int lattice_K;
  int window;           // local sweeps: d
  int stage_depth;      // global sweeps, staged variant: ring slots per warp
  int far_skip;         // FP32 global sweeps: skip chunks whose pairs stay flat
  unsigned long long* pair_count;  // global sweeps' straddle terms [formed, read], or null
  float far_cut;        // distance beyond which an FP32 term is exactly flat, plus a margin
  const double* ladder; // per-slot temperature factors (parallel tempering) or null
  int ladder_K;         // ladder size: chain c of protein p runs at T * ladder[(c - chain0) % K]
  int Lmax, nmax;       // smem sizing
  TraceRec* trace;
  int trace_chains;
  long long trace_cap;
  long long* trace_count;  // per traced chain, records written
  int* err;
  R* coords;      // per chain C-betas, 3 values per residue at 3 * (torsion offset / 2), or null
  double* tcache;  // global sweeps: per CTA (blockIdx.x) C * Lmax * 12 doubles where the FP64
                   // rebuild keeps its residue transforms between its two passes, or null
  int wait_test;  // staged sweeps: > 0 = first wait on an empty ring slot, this many tries
  // a run of whole sweeps with its own T and sigma per sweep (nsched > 0):
  // sweep q of the call (counted from the call's first proposal, which sits
  // at a sweep boundary) uses sched_T[q] and sched_sigma[q] instead of T, sigma
  int nsched;
  double sched_T[kMaxSched];
  R sched_sigma[kMaxSched];
  __device__ __forceinline__ double T_of(long long q) const { return nsched ? sched_T[q] : T; }
  __device__ __forceinline__ R sigma_of(long long q) const { return nsched ? sched_sigma[q] : sigma; }
};

// Global sweeps (Eqs. 1-3, Alg. 1 first loop) and full-energy resync.
// ST: the straddle-block rows are staged into shared memory by bulk async
// copies (stage_depth slots per warp of 32/C rows of row_bytes) instead of
// being read through L1.
template <class R, int C, bool ST>
cudaError_t launch_global(const SweepArgs<R>& a, int threads, int grid, cudaStream_t st);
template <class R, int C>
cudaError_t launch_energy(const SweepArgs<R>& a, int threads, int grid, cudaStream_t st);
template <class R, int C>
size_t global_smem_bytes(int Lmax, int nmax, int threads, int stage_depth, int row_bytes);
template <class R, int C, bool ST>
cudaError_t global_set_smem(size_t bytes);
template <class R, int C, bool ST>
cudaError_t global_occupancy(int threads, size_t smem, int* per_sm);

// Global sweeps by chain groups (FP32, far field skipped, no staging): a CTA
// holds `slots` chains of G warps each (G = 1, 2 or 4); groups of one chain.
size_t gwarp_smem_bytes(int Lmax, int slots, int G);
cudaError_t gwarp_set_smem(size_t optin);
cudaError_t gwarp_occupancy(int slots, int G, size_t smem, int* per_sm);
cudaError_t launch_gwarp(const SweepArgs<float>& a, int slots, int G, int grid, cudaStream_t st);

// Window C-betas of proposal k (window d) built by the local sweep kernel's
// window builder from one chain's torsions (device pointer theta, n values),
// in the frame of the window's first residue: out[(r - lo) * 3 + xyz].
template <class R>
cudaError_t launch_window_coords(const R* theta, int L, int k, int window, Geom<R> geom, R* out,
                                 cudaStream_t st);

// Local sweeps (Eqs. 4a-b, Eq. 6, Alg. 1 second loop).
template <class R>
cudaError_t launch_local(const SweepArgs<R>& a, int chains_per_cta, int threads, int grid,
                         cudaStream_t st);
template <class R>
size_t local_smem_bytes(int nmax, int chains_per_cta, int threads, int window);
template <class R>
cudaError_t local_set_smem(size_t bytes);

// Gradient of V for a batch of torsion vectors of one protein.
// (prot_host: host copy of the protein's record; only tab_off is read.)
// grad_set_smem raises the kernel's dynamic shared-memory limit (call once).
size_t grad_smem_bytes(size_t rsize, int L);
template <class R>
cudaError_t grad_set_smem(size_t optin);
template <class R>
cudaError_t launch_grad(const ProteinDev* prot_host, int protein, int L, const R* theta,
                        int batch, double* E_out, R* grad, Tab<R> tab, Geom<R> geom,
                        cudaStream_t st);

// Table preparation: p (or -ln p) float64 -> padded rows of (value, slope)
// pairs of R (out points at rows * Bp pairs).
template <class R>
cudaError_t launch_prep_table(const double* p, long long rows, int B, int Bp, int neglog, R* out,
                              cudaStream_t st);

// Noisy restart over all chains.
template <class R>
cudaError_t launch_noisy(const ProteinDev* prot, const int* chain_prot, int nchains, int nmax,
                         R* theta, R sd, unsigned long long seed, cudaStream_t st);

// Best-state update after a global sweep or an energy call.
template <class R>
cudaError_t launch_best(const ProteinDev* prot, const int* chain_prot, int nchains, int nmax,
                        const R* theta, R* best_theta, const double* E, double* best_E, int init,
                        cudaStream_t st);

// Conversions between the FP32 interface layout and the internal precision.
template <class R>
cudaError_t launch_convert_in(const float* src, R* dst, long long count, cudaStream_t st);
template <class R>
cudaError_t launch_convert_out(const R* src, float* dst, long long count, cudaStream_t st);

// Replica exchange between neighbouring ladder slots of parity `parity`.
template <class R>
cudaError_t launch_exchange(const ProteinDev* prot, const int* chain_prot, int nchains, int K,
                            const double* ladder, double T_scale, int parity,
                            unsigned long long seed, unsigned long long round, R* theta,
                            double* E, long long* accepted, cudaStream_t st);

cudaError_t launch_philox_fill(unsigned long long seed, unsigned chain, unsigned long long t0,
                               unsigned stream, long long count, uint4* words, float* z, float* u,
                               cudaStream_t st);

}  // namespace amh
