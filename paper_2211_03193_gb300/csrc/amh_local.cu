// amh_local.cu -- localized Metropolis sweeps (Eqs. 4a-b, Eq. 6; Alg. 1
// second loop).
//
// The proposal on torsion k is judged by V_local over residues
// [c-h, c+h], c = floor(k/2), h = floor(d/2) (Eq. 6), clipped to the chain.
// Only window pairs that straddle the pivot p(k) change distance, so
// Delta V_local sums those.  Distances inside a window depend only on the
// torsions between its residues, T(W) = [2(c-h)+1, 2(c+h)]; moves whose
// torsion index differs by a multiple of 4h have disjoint T(W), so one
// colour (all k with the same k mod 4h) is evaluated concurrently, one
// thread per window, from window-local coordinates built by NeRF in a
// frame of the window's own first residue (rigid motion leaves V_local
// unchanged).  Colours run in ascending order, k ascending within a colour.
#include "amh_internal.h"

namespace amh {

namespace {

template <class R>
struct AccT {
  using T = float;
};
template <>
struct AccT<double> {
  using T = double;
};

__host__ __device__ inline size_t align16l(size_t x) { return (x + 15) & ~size_t(15); }

template <class R>
struct LLayout {
  size_t theta, cbs, acc, total;
  __host__ __device__ LLayout(int nmax, int Gc, int threads, int window) {
    const int h = window / 2;
    size_t o = 0;
    theta = o; o = align16l(o + sizeof(R) * (size_t)nmax * Gc);
    cbs = o;   o = align16l(o + sizeof(R) * (size_t)(2 * h + 1) * 3 * threads);
    acc = o;   o = align16l(o + sizeof(unsigned long long) * Gc);
    total = o;
  }
};

// Number of torsions k in [0, n) with k = r (mod ncol).
__device__ __forceinline__ int colour_count(int n, int ncol, int r) {
  return r < n ? (n - 1 - r) / ncol + 1 : 0;
}

template <class R>
__global__ void __launch_bounds__(256) local_kernel(SweepArgs<R> a, int Gc) {
  extern __shared__ __align__(16) unsigned char smem[];
  __shared__ int s_group;
  const LLayout<R> lay(a.nmax, Gc, blockDim.x, a.window);
  R* th_s = (R*)(smem + lay.theta);          // [k][Gc]
  R* cbs = (R*)(smem + lay.cbs);             // [(j*3+xyz)][threads]
  unsigned long long* acc_s = (unsigned long long*)(smem + lay.acc);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int h = a.window / 2;
  const int ncol = 4 * h > 1 ? 4 * h : 1;
  for (;;) {
    __syncthreads();
    if (tid == 0) s_group = atomicAdd(a.queue, 1);
    __syncthreads();
    const int gi = s_group;
    if (gi >= a.ngroups) break;
    const GroupDev G = a.groups[gi];
    const ProteinDev P = a.prot[G.protein];
    const int L = P.L, n = P.n;
    for (int idx = tid; idx < n * Gc; idx += nt) {
      const int c = idx / n, k = idx - c * n;
      R v = R(0);
      if (c < G.nchains) v = a.theta[P.tors0 + (long long)(G.chain0 - P.chain0 + c) * n + k];
      th_s[k * Gc + c] = v;
    }
    if (tid < Gc) acc_s[tid] = 0ull;
    const long long t0 = a.tcount[G.chain0];
    const long long nsw = a.steps_are_sweeps ? a.steps : a.steps / n;
    __syncthreads();
    for (long long sw = 0; sw < nsw; ++sw) {
      int slot0 = 0;  // visit slot of the colour's first torsion
      for (int r = 0; r < ncol; ++r) {
        const int cnt = colour_count(n, ncol, r);
        const int items = cnt * Gc;
        for (int it = tid; it < items; it += nt) {
          const int w = it / Gc, c = it - w * Gc;
          if (c >= G.nchains) continue;
          const int k = r + w * ncol;
          const int chain = G.chain0 + c;
          const long long t = t0 + sw * n + k;
          R z, lnu;
          normal_and_lnu(draw_words(a.seed, (uint32_t)chain, (unsigned long long)t, 0u), &z,
                         &lnu);
          const R th = th_s[k * Gc + c];
          const R thn = propose(th, z, a.sigma, a.lattice_K);
          const int i = k >> 1;
          const int lo = max(0, i - h), hi = min(L - 1, i + h);
          const int p = (k + 1) >> 1;
          double dE = 0.0;
          if (p > lo && p <= hi) {
            // window-local G(s) of residues lo..hi; remember the bond axis
            V3<R> N, CA, Cc, Pax, Qax;
            first_residue(a.geom, N, CA, Cc);
            Pax = N;
            Qax = CA;
            for (int rr = lo;; ++rr) {
              const V3<R> cb = cbeta<R, true>(a.geom, N, CA, Cc);
              const int j = rr - lo;
              cbs[(j * 3 + 0) * nt + tid] = cb.x;
              cbs[(j * 3 + 1) * nt + tid] = cb.y;
              cbs[(j * 3 + 2) * nt + tid] = cb.z;
              if (rr == i) {
                if (k & 1) {  // psi_i: CA_i -> C_i
                  Pax = CA;
                  Qax = Cc;
                } else {      // phi_i: N_i -> CA_i
                  Pax = N;
                  Qax = CA;
                }
              }
              if (rr == hi) break;
              next_residue<R, true>(a.geom, N, CA, Cc, th_s[(2 * rr + 1) * Gc + c],
                                    th_s[(2 * rr + 2) * Gc + c]);
            }
            const Aff<R> A = rotation(Pax, Qax, wrap_angle(thn - th));
            typename AccT<R>::T acc = 0;
            const auto* tab = a.tab.E + P.tab_off;
            for (int b = p; b <= hi; ++b) {
              const int jb = b - lo;
              const V3<R> xb = v3<R>(cbs[(jb * 3 + 0) * nt + tid], cbs[(jb * 3 + 1) * nt + tid],
                                     cbs[(jb * 3 + 2) * nt + tid]);
              const V3<R> yb = apply(A, xb);
              for (int aa = lo; aa < p; ++aa) {
                const int ja = aa - lo;
                const V3<R> xa = v3<R>(cbs[(ja * 3 + 0) * nt + tid],
                                       cbs[(ja * 3 + 1) * nt + tid],
                                       cbs[(ja * 3 + 2) * nt + tid]);
                const auto* row = tab + (long long)row_of(L, aa, b) * a.tab.Bp;
                acc += pair_term(row, dist_(xa, yb), a.tab) - pair_term(row, dist_(xa, xb), a.tab);
              }
            }
            dE = (double)acc;
          }
          const double Tc = a.ladder ? a.T * a.ladder[(chain - P.chain0) % a.ladder_K] : a.T;
          const int accept = (double)lnu < -dE / Tc;
          if (accept) {
            th_s[k * Gc + c] = thn;
            atomicAdd(&acc_s[c], 1ull);
          }
          const long long v = t0 + sw * n + slot0 + w;
          if (chain < a.trace_chains && v < a.trace_cap) {
            TraceRec rec;
            rec.k = k;
            rec.accept = accept;
            rec.theta_new = (double)thn;
            rec.lnu = (double)lnu;
            rec.dE = dE;
            a.trace[(size_t)chain * a.trace_cap + v] = rec;
          }
        }
        slot0 += cnt;
        __syncthreads();
      }
    }
    const long long t_end = t0 + nsw * n;
    for (int idx = tid; idx < n * Gc; idx += nt) {
      const int c = idx / n, k = idx - c * n;
      if (c >= G.nchains) continue;
      a.theta[P.tors0 + (long long)(G.chain0 - P.chain0 + c) * n + k] = th_s[k * Gc + c];
    }
    if (tid < Gc && tid < G.nchains) {
      const int chain = G.chain0 + tid;
      a.tcount[chain] = t_end;
      if (a.acc_out) a.acc_out[chain] = (long long)acc_s[tid];
      if (a.trace_count && chain < a.trace_chains)
        a.trace_count[chain] = t_end < a.trace_cap ? t_end : a.trace_cap;
    }
  }
}

}  // namespace

template <class R>
size_t local_smem_bytes(int nmax, int chains_per_cta, int threads, int window) {
  return LLayout<R>(nmax, chains_per_cta, threads, window).total;
}

template <class R>
cudaError_t local_set_smem(size_t optin) {
  return allow_dynamic_smem(local_kernel<R>, optin);
}

template <class R>
cudaError_t launch_local(const SweepArgs<R>& a, int chains_per_cta, int threads, int grid,
                         cudaStream_t st) {
  const size_t sm = local_smem_bytes<R>(a.nmax, chains_per_cta, threads, a.window);
  local_kernel<R><<<grid, threads, sm, st>>>(a, chains_per_cta);
  return cudaGetLastError();
}

template size_t local_smem_bytes<float>(int, int, int, int);
template size_t local_smem_bytes<double>(int, int, int, int);
template cudaError_t local_set_smem<float>(size_t);
template cudaError_t local_set_smem<double>(size_t);
template cudaError_t launch_local<float>(const SweepArgs<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_local<double>(const SweepArgs<double>&, int, int, int, cudaStream_t);

}  // namespace amh
