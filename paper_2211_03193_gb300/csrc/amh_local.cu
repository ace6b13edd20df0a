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
// thread per window, from window-local coordinates in the frame of the
// window's own first residue (rigid motion leaves V_local unchanged).
// Colours run in ascending order, k ascending within a colour.
//
// Window coordinates come from residue transforms: with ideal geometry
// residue i sits at T_{lo+1} o ... o T_i applied to a canonical residue in
// the frame of residue lo, and T_i depends on (psi_{i-1}, phi_i) only (in
// FP32 from the bilinear (1, cos, sin) basis of residue_basis: two sincos
// and 108 FMA).  The CTA keeps every T_i of its chains in shared memory and
// recomputes T_p(k) when move k is accepted; T_p(k) belongs to the window of
// move k alone within a colour.  Each window draws its proposal's Philox
// words itself (they depend on the counter only).
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

__host__ __device__ inline size_t align32l(size_t x) { return (x + 31) & ~size_t(31); }

template <class R>
struct LLayout {
  size_t kb, theta, tr, cbs, acc, total;
  __host__ __device__ LLayout(int nmax, int Gc, int threads, int window) {
    const int h = window / 2;
    const int Lmax = nmax / 2;
    size_t o = 0;
    kb = o;    o = align32l(o + sizeof(double) * 216);  // FP64 basis (scratch), FP32 copy after
    theta = o; o = align32l(o + sizeof(R) * (size_t)nmax * Gc);
    tr = o;    o = align32l(o + sizeof(Pt4<R>) * 3 * (size_t)Lmax * Gc);
    cbs = o;   o = align32l(o + sizeof(R) * (size_t)(2 * h + 1) * 3 * threads);
    acc = o;   o = align32l(o + sizeof(unsigned long long) * Gc);
    total = o;
  }
};

// T_i of residue i from (psi_{i-1}, phi_i): the FP32 form takes the
// bilinear basis of residue_basis rounded to FP32 (two sincos and 108 FMA),
// the FP64 form NeRF in FP64.
__device__ __forceinline__ Aff<float> local_step(const Geom<float>&, const CanonicalResidue<float>&,
                                                 const float* kbf, float psi, float phi) {
  float sp, cp, sf, cf;
  sincosf(psi, &sp, &cp);
  sincosf(phi, &sf, &cf);
  const float f[3] = {1.f, cp, sp}, gg[3] = {1.f, cf, sf};
  float v[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) v[q] = 0.f;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const float w = f[a] * gg[b];
      const float* K = kbf + (a * 3 + b) * 12;
#pragma unroll
      for (int q = 0; q < 12; ++q) v[q] = fmaf(w, K[q], v[q]);
    }
  Aff<float> T;
#pragma unroll
  for (int q = 0; q < 9; ++q) T.m[q] = v[q];
#pragma unroll
  for (int q = 0; q < 3; ++q) T.t[q] = v[9 + q];
  return T;
}
__device__ __forceinline__ Aff<double> local_step(const Geom<double>& g,
                                                  const CanonicalResidue<double>& cr,
                                                  const float*, double psi, double phi) {
  return residue_step(g, cr, psi, phi);
}

// Number of torsions k in [0, n) with k = r (mod ncol).
__device__ __forceinline__ int colour_count(int n, int ncol, int r) {
  return r < n ? (n - 1 - r) / ncol + 1 : 0;
}

// Pair term through the texture path (FP32) or the table rows (FP64).
template <class R>
__device__ __forceinline__ R local_term(const Tab<R>& tb, long long tab_off, int row, R d);
template <>
__device__ __forceinline__ float local_term<float>(const Tab<float>& tb, long long tab_off,
                                                   int row, float d) {
  if (tb.tex) return pair_term_tex((int)tab_off + row * tb.Bp, d, tb);
  return pair_term(tb.E + tab_off + (long long)row * tb.Bp, d, tb);
}
template <>
__device__ __forceinline__ double local_term<double>(const Tab<double>& tb, long long tab_off,
                                                     int row, double d) {
  return pair_term(tb.E + tab_off + (long long)row * tb.Bp, d, tb);
}

// Delta V_local of a window's pairs on the texture path (FP32): for each
// downstream atom b, the upstream atoms a in [lo, p) up to NA at a time with
// no branch, so a thread keeps 2 NA fetches in flight (a loop over a waits
// for each pair's fetches in turn).  Slots past p, and pairs at or past the
// last bin centre both before and after the move, read nothing and add
// 0 - 0; the terms are added in the order of the plain loop below, so the
// sum is the same bit for bit.  cbs: the window's C-betas, [(j*3+xyz)][nt].
// NA is the smallest of 3, 5, 8 that holds h + 1 >= p - lo (d up to 14).
constexpr int kLA = 8;

template <int NA>
__device__ __forceinline__ float window_pairs_tex(const float* cbs, int nt, int tid, int L,
                                                  int lo, int p, int hi, const Aff<float>& A,
                                                  const Tab<float>& tb, long long tab_off) {
  const int na = p - lo;
  // the upstream atoms and the entry index of their pairs with b = p, once:
  // r(a, b + 1) = r(a, b) + 1
  V3<float> xa[NA];
  int re[NA];
#pragma unroll
  for (int q = 0; q < NA; ++q) {
    const int jq = q < na ? q : 0;
    xa[q] = v3<float>(cbs[(jq * 3 + 0) * nt + tid], cbs[(jq * 3 + 1) * nt + tid],
                      cbs[(jq * 3 + 2) * nt + tid]);
    re[q] = (int)tab_off + row_of(L, lo + jq, p) * tb.Bp;
  }
  float acc = 0.f;
  for (int b = p; b <= hi; ++b) {
    const int jb = b - lo;
    const V3<float> xb = v3<float>(cbs[(jb * 3 + 0) * nt + tid], cbs[(jb * 3 + 1) * nt + tid],
                                   cbs[(jb * 3 + 2) * nt + tid]);
    const V3<float> yb = apply(A, xb);
    const int db = (b - p) * tb.Bp;
#pragma unroll
    for (int q = 0; q < NA; ++q) {
      const unsigned ok = q < na;
      const float u1 = bin_sat(dist_fast(xa[q], yb), tb), u0 = bin_sat(dist_fast(xa[q], xb), tb);
      const unsigned need = ok & (fminf(u0, u1) < 1.f);
      acc += term_tex_if(re[q] + db, u1, tb, need) - term_tex_if(re[q] + db, u0, tb, need);
    }
  }
  return acc;
}

// The window builder: residue rr of [lo, hi] sits at M_rr = T_{lo+1} o ...
// o T_rr applied to the canonical residue (the frame of residue lo); Ti(rr)
// gives T_rr and emit(rr, M_rr) receives each residue's map in order.
template <class R, class TI, class EMIT>
__device__ __forceinline__ void window_walk(int lo, int hi, TI Ti, EMIT emit) {
  Aff<R> M = identity_map<R>();
  for (int rr = lo; rr <= hi; ++rr) {
    if (rr > lo) M = compose(M, Ti(rr));
    emit(rr, M);
  }
}

template <class R>
__global__ void __launch_bounds__(256) local_kernel(SweepArgs<R> a, int Gc) {
  extern __shared__ __align__(32) unsigned char smem[];
  __shared__ int s_group;
  const LLayout<R> lay(a.nmax, Gc, blockDim.x, a.window);
  double* kb = (double*)(smem + lay.kb);     // residue-transform basis (FP64; FP32 copy at kb+108)
  R* th_s = (R*)(smem + lay.theta);          // [k][Gc]
  Pt4<R>* tr_s = (Pt4<R>*)(smem + lay.tr);   // [i][Gc][3]: T_i, i >= 1
  R* cbs = (R*)(smem + lay.cbs);             // [(j*3+xyz)][threads]
  unsigned long long* acc_s = (unsigned long long*)(smem + lay.acc);
  const int tid = threadIdx.x, nt = blockDim.x;
  const int h = a.window / 2;
  const int ncol = 4 * h > 1 ? 4 * h : 1;
  const CanonicalResidue<R> cr = canonical_residue(a.geom);
  residue_basis(a.geom64, kb);
  // its FP32 copy over the FP64 scratch half (kb[108..216) as 108 floats)
  float* kbf = reinterpret_cast<float*>(kb + 108);
  for (int q = tid; q < 108; q += nt) kbf[q] = (float)kb[q];
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
    // accepted moves counted per thread and added once per call: when the
    // block size is a multiple of Gc every item of a thread belongs to chain
    // slot tid % Gc (one shared atomic per acceptance serialised the
    // accepting windows of a chain)
    const bool own_slot = nt % Gc == 0;
    unsigned nacc = 0;
    __syncthreads();
    for (int idx = tid; idx < (L - 1) * Gc; idx += nt) {
      const int i = 1 + idx / Gc, c = idx % Gc;
      aff_store4(tr_s + ((size_t)i * Gc + c) * 3,
                 local_step(a.geom, cr, kbf, th_s[(2 * i - 1) * Gc + c], th_s[2 * i * Gc + c]));
    }
    const long long t0 = a.tcount[G.chain0];
    const long long nsw = a.steps_are_sweeps ? a.steps : a.steps / n;
    __syncthreads();
    for (long long sw = 0; sw < nsw; ++sw) {
      const R sig = a.sigma_of(sw);
      const double Tsw = a.T_of(sw);
      int slot0 = 0;  // visit slot of the colour's first torsion
      for (int r = 0; r < ncol; ++r) {
        const int cnt = colour_count(n, ncol, r);
        const int items = cnt * Gc;
        for (int it = tid; it < items; it += nt) {
          const int w = it / Gc, c = it - w * Gc;
          if (c >= G.nchains) continue;
          const int k = r + w * ncol;
          const int chain = G.chain0 + c;
          // the proposal's draws (they depend on the counter only)
          R z, lnu;
          normal_and_lnu(draw_words(a.seed, (uint32_t)chain, (unsigned long long)(t0 + sw * n + k),
                                    0u),
                         &z, &lnu);
          const R th = th_s[k * Gc + c];
          const R thn = propose(th, z, sig, a.lattice_K);
          const int i = k >> 1;
          const int lo = max(0, i - h), hi = min(L - 1, i + h);
          const int p = (k + 1) >> 1;
          typename AccT<R>::T acc = 0;
          const bool scored = p > lo && p <= hi;
          Aff<R> A;  // the move
          if (scored) {
            // window coordinates from the cached residue transforms;
            // remember the bond axis
            V3<R> Pax = cr.N, Qax = cr.CA;
            window_walk<R>(
                lo, hi, [&](int rr) { return aff_load4(tr_s + ((size_t)rr * Gc + c) * 3); },
                [&](int rr, const Aff<R>& M) {
                  const V3<R> cb = apply(M, cr.CB);
                  const int j = rr - lo;
                  cbs[(j * 3 + 0) * nt + tid] = cb.x;
                  cbs[(j * 3 + 1) * nt + tid] = cb.y;
                  cbs[(j * 3 + 2) * nt + tid] = cb.z;
                  if (rr == i) {
                    if (k & 1) {  // psi_i: CA_i -> C_i
                      Pax = apply(M, cr.CA);
                      Qax = apply(M, cr.C);
                    } else {      // phi_i: N_i -> CA_i
                      Pax = apply(M, cr.N);
                      Qax = apply(M, cr.CA);
                    }
                  }
                });
            A = rotation(Pax, Qax, wrap_angle(thn - th));
            bool done = false;
            if constexpr (sizeof(R) == 4) {
              if (a.tab.tex && h + 1 <= kLA) {
                acc = h + 1 <= 3   ? window_pairs_tex<3>(cbs, nt, tid, L, lo, p, hi, A, a.tab,
                                                         P.tab_off)
                      : h + 1 <= 5 ? window_pairs_tex<5>(cbs, nt, tid, L, lo, p, hi, A, a.tab,
                                                         P.tab_off)
                                   : window_pairs_tex<kLA>(cbs, nt, tid, L, lo, p, hi, A, a.tab,
                                                           P.tab_off);
                done = true;
              }
            }
            // the plain loop: FP64, table entries through L1, or windows past d = 14
            for (int b = p; b <= hi && !done; ++b) {
              const int jb = b - lo;
              const V3<R> xb = v3<R>(cbs[(jb * 3 + 0) * nt + tid], cbs[(jb * 3 + 1) * nt + tid],
                                     cbs[(jb * 3 + 2) * nt + tid]);
              const V3<R> yb = apply(A, xb);
              // rows (aa, b), aa ascending: r(aa+1, b) - r(aa, b) = L - aa - 2
              int row = row_of(L, lo, b);
              for (int aa = lo; aa < p; ++aa) {
                const int ja = aa - lo;
                const V3<R> xa = v3<R>(cbs[(ja * 3 + 0) * nt + tid],
                                       cbs[(ja * 3 + 1) * nt + tid],
                                       cbs[(ja * 3 + 2) * nt + tid]);
                acc += local_term(a.tab, P.tab_off, row, dist_fast(xa, yb)) -
                       local_term(a.tab, P.tab_off, row, dist_fast(xa, xb));
                row += L - aa - 2;
              }
            }
          }
          const double dE = (double)acc;
          const double Tc = a.ladder ? Tsw * a.ladder[(chain - P.chain0) % a.ladder_K] : Tsw;
          // ln u < -dE / T with T > 0 (FP32 form: in FP32, the precision of dE)
          const int accept = sizeof(R) == 4 ? (float)lnu * (float)Tc < -(float)acc
                                            : (double)lnu * Tc < -dE;
          if (accept) {
            th_s[k * Gc + c] = thn;
            if (own_slot)
              ++nacc;
            else
              atomicAdd(&acc_s[c], 1ull);
            // T_p depends on torsions 2p-1 and 2p, one of which is k: rebuilt
            // from them (composing the move into T_p instead lost ~1e-6 of
            // orthonormality per update, ~1e-3 in later Delta-E)
            if (p >= 1 && p < L)
              aff_store4(tr_s + ((size_t)p * Gc + c) * 3,
                         local_step(a.geom, cr, kbf, th_s[(2 * p - 1) * Gc + c],
                                    th_s[2 * p * Gc + c]));
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
    if (own_slot && nacc) atomicAdd(&acc_s[tid % Gc], (unsigned long long)nacc);
    __syncthreads();
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

// One window's C-betas by the local kernel's builder: the residue
// transforms as the kernel caches them (local_step of the torsions, stored
// and loaded through the same 4-value layout), composed by window_walk in
// thread 0 (the CTA's 32 threads first form the basis, as the kernel does).
template <class R>
__global__ void window_coords_kernel(const R* theta, int L, int k, int window, Geom<R> g,
                                     Geom<double> g64, R* out) {
  __shared__ double kb[216];
  residue_basis(g64, kb);
  float* kbf = reinterpret_cast<float*>(kb + 108);
  for (int q = threadIdx.x; q < 108; q += blockDim.x) kbf[q] = (float)kb[q];
  __syncthreads();
  if (threadIdx.x != 0 || blockIdx.x != 0) return;
  const CanonicalResidue<R> cr = canonical_residue(g);
  const int h = window / 2, i = k >> 1;
  const int lo = max(0, i - h), hi = min(L - 1, i + h);
  window_walk<R>(
      lo, hi,
      [&](int rr) {
        Pt4<R> q[3];
        aff_store4(q, local_step(g, cr, kbf, theta[2 * rr - 1], theta[2 * rr]));
        return aff_load4(q);
      },
      [&](int rr, const Aff<R>& M) {
        const V3<R> cb = apply(M, cr.CB);
        out[(rr - lo) * 3 + 0] = cb.x;
        out[(rr - lo) * 3 + 1] = cb.y;
        out[(rr - lo) * 3 + 2] = cb.z;
      });
}

}  // namespace

template <class R>
cudaError_t launch_window_coords(const R* theta, int L, int k, int window, Geom<R> geom, R* out,
                                 cudaStream_t st) {
  window_coords_kernel<R><<<1, 32, 0, st>>>(theta, L, k, window, geom,
                                             ideal_geometry<double>(), out);
  return cudaGetLastError();
}
template cudaError_t launch_window_coords<float>(const float*, int, int, int, Geom<float>, float*,
                                                 cudaStream_t);
template cudaError_t launch_window_coords<double>(const double*, int, int, int, Geom<double>,
                                                  double*, cudaStream_t);

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
