// amh_misc.cu -- gradient of V, table preparation, noisy restart, best-state
// bookkeeping, precision conversions and the Philox fill used for checking.
#include "amh_internal.h"

namespace amh {

// Shared memory of one gradient CTA (256 threads): coordinates and partial
// forces in R, suffix sums in FP64, and the chain-building scan's warp
// totals.
// Parts of the a range per pair-force item (partial forces kept apart so
// the sum needs no atomics and its order is fixed).
constexpr int kGradParts = 4;

size_t grad_smem_bytes(size_t rsize, int L) {
  return ((rsize * (12 + 3 * kGradParts) * L + 15) & ~(size_t)15) + sizeof(double) * 6 * (L + 1) +
         sizeof(double) * (12 * 8 + 216);
}

// The residue-transform cache (12 doubles per residue) is used when it fits.
static size_t grad_cache_bytes(int L) { return sizeof(double) * 12 * (size_t)L; }

namespace {

// ---------------------------------------------------------------- gradient
// dV/ds_k for one torsion vector per CTA.  Changing s_k turns every C-beta
// b >= p(k) about the bond axis (u, o), so dV/ds_k = sum_{b>=p} g_b .
// (u x (x_b - o)) = u . (M_p - o x G_p) with g_b = dV/dx_b (pair forces),
// G_p = sum_{b>=p} g_b, M_p = sum_{b>=p} x_b x g_b.  Pairs on the same side
// of the pivot contribute forces that cancel in the sum.
constexpr int kGradThreads = 256;

// Suffix sums (over b >= p) of six FP64 values, one block of residues per
// thread, scanned across the CTA.  wtot: 8 warps x 6 doubles of scratch.
__device__ void suffix_scan6(int L, const float* CBf, const double* CBd, const float* gbf,
                             const double* gbd, double* GM, double* wtot) {
  const int tid = threadIdx.x, nt = blockDim.x, lane = tid & 31, warp = tid >> 5;
  const int nb = (L + nt - 1) / nt;
  // thread t owns residues [L - (t+1) nb, L - t nb): reversed order, so an
  // inclusive prefix over threads is a suffix over residues
  const int hi = L - tid * nb, lo = max(0, hi - nb);
  double v[6] = {0, 0, 0, 0, 0, 0};
  for (int b = hi - 1; b >= lo; --b) {
    const double x0 = CBf ? CBf[3 * b] : CBd[3 * b], x1 = CBf ? CBf[3 * b + 1] : CBd[3 * b + 1],
                 x2 = CBf ? CBf[3 * b + 2] : CBd[3 * b + 2];
    const double g0 = gbf ? gbf[3 * b] : gbd[3 * b], g1 = gbf ? gbf[3 * b + 1] : gbd[3 * b + 1],
                 g2 = gbf ? gbf[3 * b + 2] : gbd[3 * b + 2];
    v[0] += g0; v[1] += g1; v[2] += g2;
    v[3] += x1 * g2 - x2 * g1; v[4] += x2 * g0 - x0 * g2; v[5] += x0 * g1 - x1 * g0;
  }
  double incl[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) incl[q] = v[q];
  for (int off = 1; off < 32; off <<= 1) {
#pragma unroll
    for (int q = 0; q < 6; ++q) {
      const double o = __shfl_up_sync(0xffffffffu, incl[q], off);
      if (lane >= off) incl[q] += o;
    }
  }
  if (lane == 31)
#pragma unroll
    for (int q = 0; q < 6; ++q) wtot[warp * 6 + q] = incl[q];
  __syncthreads();
  double base[6] = {0, 0, 0, 0, 0, 0};
  for (int w = 0; w < warp; ++w)
#pragma unroll
    for (int q = 0; q < 6; ++q) base[q] += wtot[w * 6 + q];
  // running suffix sum at the top of this thread's block
  double run[6];
#pragma unroll
  for (int q = 0; q < 6; ++q) run[q] = base[q] + incl[q] - v[q];
  double* r = GM + (size_t)L * 6;
  if (tid == 0)
#pragma unroll
    for (int q = 0; q < 6; ++q) r[q] = 0.0;
  for (int b = hi - 1; b >= lo; --b) {
    const double x0 = CBf ? CBf[3 * b] : CBd[3 * b], x1 = CBf ? CBf[3 * b + 1] : CBd[3 * b + 1],
                 x2 = CBf ? CBf[3 * b + 2] : CBd[3 * b + 2];
    const double g0 = gbf ? gbf[3 * b] : gbd[3 * b], g1 = gbf ? gbf[3 * b + 1] : gbd[3 * b + 1],
                 g2 = gbf ? gbf[3 * b + 2] : gbd[3 * b + 2];
    run[0] += g0; run[1] += g1; run[2] += g2;
    run[3] += x1 * g2 - x2 * g1; run[4] += x2 * g0 - x0 * g2; run[5] += x0 * g1 - x1 * g0;
    double* o = GM + (size_t)b * 6;
#pragma unroll
    for (int q = 0; q < 6; ++q) o[q] = run[q];
  }
}

template <class R>
__global__ void __launch_bounds__(kGradThreads) grad_kernel(int L, long long tab_off,
                                                            const R* __restrict__ theta,
                                                            double* __restrict__ E_out,
                                                            R* __restrict__ grad, Tab<R> tb,
                                                            Geom<double> geom, int use_cache) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int n = 2 * L;
  R* X = (R*)smem;          // [4][L][3]: N, CA, C, CB
  R* gb = X + 12 * L;       // [kGradParts][L][3] partial dV/dx_b (parts of the a range)
  double* GM = (double*)(smem + (((size_t)sizeof(R) * (12 + 3 * kGradParts) * L + 15) &
                                 ~(size_t)15));  // [L+1][6]
  double* scan = GM + (size_t)6 * (L + 1);  // [8][12] warp totals of the chain-building scan
  double* kb = scan + 8 * 12;               // [216] residue-transform basis
  double* cache = kb + 216;                 // [L][12] residue transforms (if use_cache)
  __shared__ double wpart[64];  // warp energy partials, then the suffix scan's 8 x 6 totals
  const int v = blockIdx.x, tid = threadIdx.x, nt = blockDim.x;
  const R* th = theta + (size_t)v * n;
  // G(s) built in FP64 by one warp (FP64 is the scarce pipe: a wider scan
  // composes more transforms in all), stored in R as the sweeps' resync does
  residue_basis(geom, kb);
  if (tid < 32)
    build_chains_scan(
        geom, kb, L, 1, [&](int, int k) { return (double)th[k]; },
        [&](int, int i, V3<double> N, V3<double> CA, V3<double> Cc, V3<double> CB) {
          const V3<double> at[4] = {N, CA, Cc, CB};
#pragma unroll
          for (int q = 0; q < 4; ++q) {
            X[(q * L + i) * 3 + 0] = (R)at[q].x;
            X[(q * L + i) * 3 + 1] = (R)at[q].y;
            X[(q * L + i) * 3 + 2] = (R)at[q].z;
          }
        },
        scan, use_cache ? cache : nullptr, 32);
  __syncthreads();
  const R* CB = X + 9 * L;
  // pair forces: item (b, q) sums over a in part q of [0, L); each pair is
  // visited from both ends, so no atomics are needed.  Rows advance
  // incrementally: r(a+1, b) - r(a, b) = L - a - 2 below b, +1 above it.
  double esum = 0.0;
  const int chunk = (L + kGradParts - 1) / kGradParts;
  for (int it = tid; it < kGradParts * L; it += nt) {
    const int b = it / kGradParts, q = it - b * kGradParts;
    const int a0 = min(L, q * chunk), a1 = min(L, a0 + chunk);
    const V3<R> xb = v3<R>(CB[3 * b], CB[3 * b + 1], CB[3 * b + 2]);
    R gx = 0, gy = 0, gz = 0;
    R epart = 0;
    // dV/dx_b from pair (a, b): e'(d) (x_b - x_a) / d, 1/d from one rsqrt
    auto pair = [&](int a, const typename Vec2<R>::T* row) -> R {
      const V3<R> dlt = xb - v3<R>(CB[3 * a], CB[3 * a + 1], CB[3 * a + 2]);
      const R d2 = fma(dlt.z, dlt.z, fma(dlt.y, dlt.y, fma(dlt.x, dlt.x, R(1e-30))));
      const R inv = rsqrt_(d2);
      R sl;
      const R e = pair_term_slope(row, d2 * inv, tb, &sl);
      const R f = sl * inv;
      gx += f * dlt.x;
      gy += f * dlt.y;
      gz += f * dlt.z;
      return e;
    };
    const int e1 = min(a1, b);
    if (a0 < e1) {
      const auto* row = tb.E + tab_off + (long long)row_of(L, a0, b) * tb.Bp;
#pragma unroll 4
      for (int a = a0; a < e1; ++a) {
        epart += pair(a, row);
        row += (long long)(L - a - 2) * tb.Bp;
      }
    }
    const int s2 = max(a0, b + 1);
    if (s2 < a1) {
      const auto* row = tb.E + tab_off + (long long)row_of(L, b, s2) * tb.Bp;
#pragma unroll 4
      for (int a = s2; a < a1; ++a, row += tb.Bp) pair(a, row);
    }
    R* gp = gb + ((size_t)q * L + b) * 3;
    gp[0] = gx;
    gp[1] = gy;
    gp[2] = gz;
    esum += (double)epart;
  }
  for (int off = 16; off > 0; off >>= 1) esum += __shfl_xor_sync(0xffffffffu, esum, off);
  if ((tid & 31) == 0) wpart[tid >> 5] = esum;
  __syncthreads();
  // fold the parts in order: g_b in part 0 of gb
  for (int q = tid; q < 3 * L; q += nt) {
    R g = gb[q];
#pragma unroll
    for (int h = 1; h < kGradParts; ++h) g += gb[(size_t)h * 3 * L + q];
    gb[q] = g;
  }
  if (tid == 0) {
    double e = 0.0;
    for (int w = 0; w < (nt >> 5); ++w) e += wpart[w];
    E_out[v] = e;
  }
  __syncthreads();
  if (sizeof(R) == 4)
    suffix_scan6(L, (const float*)CB, nullptr, (const float*)gb, nullptr, GM, wpart);
  else
    suffix_scan6(L, nullptr, (const double*)CB, nullptr, (const double*)gb, GM, wpart);
  __syncthreads();
  for (int k = tid; k < n; k += nt) {
    const int i = k >> 1, p = (k + 1) >> 1;
    double val = 0.0;
    if (k != 0 && p < L) {
      const int qa = (k & 1) ? 1 : 0, qb = (k & 1) ? 2 : 1;  // psi: CA->C, phi: N->CA
      const double o0 = X[(qa * L + i) * 3], o1 = X[(qa * L + i) * 3 + 1], o2 = X[(qa * L + i) * 3 + 2];
      double u0 = X[(qb * L + i) * 3] - o0, u1 = X[(qb * L + i) * 3 + 1] - o1,
             u2 = X[(qb * L + i) * 3 + 2] - o2;
      const double un = rsqrt(u0 * u0 + u1 * u1 + u2 * u2);
      u0 *= un; u1 *= un; u2 *= un;
      const double* r = GM + (size_t)p * 6;
      const double t0 = r[3] - (o1 * r[2] - o2 * r[1]);
      const double t1 = r[4] - (o2 * r[0] - o0 * r[2]);
      const double t2 = r[5] - (o0 * r[1] - o1 * r[0]);
      val = u0 * t0 + u1 * t1 + u2 * t2;
    }
    grad[(size_t)v * n + k] = (R)val;
  }
}

// ---------------------------------------------------------------- table
// Entry j of a row, E = -ln max(p, 1e-300) and D_j = E_{j+1} - E_j: (E_j,
// D_j) in FP64, (E_j - j D_j, (B-1) D_j) in FP32 (the layouts of Tab); the
// last bin and the padding hold (E_{B-1}, 0).
__device__ __forceinline__ double neglog_p(double q, int neglog) {
  return neglog ? q : -log(q > 1e-300 ? q : 1e-300);
}

template <class R>
__global__ void prep_table_kernel(const double* __restrict__ p, long long rows, int B, int Bp,
                                  int neglog, typename Vec2<R>::T* __restrict__ out) {
  const long long total = rows * Bp;
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < total;
       i += (long long)gridDim.x * blockDim.x) {
    const long long r = i / Bp;
    const int j = (int)(i - r * Bp);
    const double* pr = p + r * B;
    const double e0 = neglog_p(pr[j < B ? j : B - 1], neglog);
    const double e1 = j + 1 < B ? neglog_p(pr[j + 1], neglog) : e0;
    typename Vec2<R>::T v;
    if (sizeof(R) == 8) {  // (E_j, D_j)
      v.x = (R)e0;
      v.y = (R)(e1 - e0);
    } else {               // (E_j - j D_j, (B-1) D_j): see Tab
      const double D = e1 - e0;
      v.x = (R)(e0 - (double)j * D);
      v.y = (R)((double)(B - 1) * D);
    }
    out[i] = v;
  }
}

// ---------------------------------------------------------------- noisy restart
template <class R>
__global__ void noisy_kernel(const ProteinDev* __restrict__ prot, const int* __restrict__ chain_prot,
                             R* __restrict__ theta, R sd, unsigned long long seed) {
  const int chain = blockIdx.y;
  const ProteinDev P = prot[chain_prot[chain]];
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= P.n) return;
  R z, lnu;
  normal_and_lnu(draw_words(seed, (uint32_t)chain, (unsigned long long)k, 1u), &z, &lnu);
  R* th = theta + P.tors0 + (long long)(chain - P.chain0) * P.n;
  th[k] = wrap_angle(th[k] + sd * z);
}

// ---------------------------------------------------------------- best state
template <class R>
__global__ void best_kernel(const ProteinDev* __restrict__ prot, const int* __restrict__ chain_prot,
                            const R* __restrict__ theta, R* __restrict__ best_theta,
                            const double* __restrict__ E, double* __restrict__ best_E, int init) {
  const int chain = blockIdx.x;
  const ProteinDev P = prot[chain_prot[chain]];
  __shared__ int better;
  if (threadIdx.x == 0) {
    better = init || E[chain] < best_E[chain];
    if (better) best_E[chain] = E[chain];
  }
  __syncthreads();
  if (!better) return;
  const long long off = P.tors0 + (long long)(chain - P.chain0) * P.n;
  for (int k = threadIdx.x; k < P.n; k += blockDim.x) best_theta[off + k] = theta[off + k];
}

// ---------------------------------------------------------------- replica exchange
// One warp per candidate pair (slots j, j+1 of a ladder, j = parity mod 2):
// swap the two states iff ln u < (1/T_j - 1/T_{j+1}) (E_j - E_{j+1}), u from
// Philox stream 3 at (chain of slot j, round).  Energies must be current.
template <class R>
__global__ void exchange_kernel(const ProteinDev* __restrict__ prot,
                                const int* __restrict__ chain_prot, int nchains, int K,
                                const double* __restrict__ ladder, double T_scale, int parity,
                                unsigned long long seed, unsigned long long round,
                                R* __restrict__ theta, double* __restrict__ E,
                                long long* __restrict__ accepted) {
  const int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5, lane = threadIdx.x & 31;
  const int a = warp;  // candidate lower slot = chain a
  if (a >= nchains) return;
  const ProteinDev P = prot[chain_prot[a]];
  const int j = (a - P.chain0) % K;
  int swap = 0;
  const bool cand = ((j & 1) == parity) && (j + 1 < K);
  if (cand) {
    const int b = a + 1;
    if (lane == 0) {
      const uint4 w = draw_words(seed, (uint32_t)a, round, 3u);
      const double lnu = log(uniform23d(w.x));
      const double delta = (1.0 / (T_scale * ladder[j]) - 1.0 / (T_scale * ladder[j + 1])) *
                           (E[a] - E[b]);
      swap = lnu < delta;
    }
    swap = __shfl_sync(0xffffffffu, swap, 0);
    if (swap) {
      R* ta = theta + P.tors0 + (long long)(a - P.chain0) * P.n;
      R* tb = theta + P.tors0 + (long long)(b - P.chain0) * P.n;
      for (int k = lane; k < P.n; k += 32) {
        const R q = ta[k];
        ta[k] = tb[k];
        tb[k] = q;
      }
      if (lane == 0) {
        const double q = E[a];
        E[a] = E[b];
        E[b] = q;
      }
    }
  }
  if (lane == 0 && accepted) {
    // each chain is written once: by its own warp (as the lower slot)
    accepted[a] = swap;
  }
}

// ---------------------------------------------------------------- conversions
template <class R>
__global__ void convert_in_kernel(const float* __restrict__ src, R* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (R)src[i];
}
template <class R>
__global__ void convert_out_kernel(const R* __restrict__ src, float* __restrict__ dst, long long n) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n;
       i += (long long)gridDim.x * blockDim.x)
    dst[i] = (float)src[i];
}

// ---------------------------------------------------------------- Philox fill
__global__ void philox_kernel(unsigned long long seed, unsigned chain, unsigned long long t0,
                              unsigned stream, long long count, uint4* words, float* z, float* u) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    const uint4 w = draw_words(seed, chain, t0 + (unsigned long long)i, stream);
    words[i] = w;
    float zz, ll;
    normal_and_lnu(w, &zz, &ll);
    if (z) z[i] = zz;
    if (u) u[i] = uniform23f(w.z);
  }
}

inline int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  if (g > 65535LL * 8) g = 65535LL * 8;
  return (int)(g > 0 ? g : 1);
}

}  // namespace

template <class R>
cudaError_t grad_set_smem(size_t optin) {
  return allow_dynamic_smem(grad_kernel<R>, optin);
}

template <class R>
cudaError_t launch_grad(const ProteinDev* prot_host, int protein, int L, const R* theta, int batch,
                        double* E_out, R* grad, Tab<R> tab, Geom<R> geom, cudaStream_t st) {
  (void)protein;
  size_t sm = grad_smem_bytes(sizeof(R), L);
  if (batch <= 0) return cudaSuccess;
  (void)geom;
  int dev = 0, optin = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const int use_cache = sm + grad_cache_bytes(L) + 1024 <= (size_t)optin ? 1 : 0;
  if (use_cache) sm += grad_cache_bytes(L);
  grad_kernel<R><<<batch, kGradThreads, sm, st>>>(L, prot_host->tab_off, theta, E_out, grad, tab,
                                                  ideal_geometry<double>(), use_cache);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_prep_table(const double* p, long long rows, int B, int Bp, int neglog, R* out,
                              cudaStream_t st) {
  if (rows <= 0) return cudaSuccess;
  prep_table_kernel<R><<<grid_for(rows * Bp, 256), 256, 0, st>>>(
      p, rows, B, Bp, neglog, reinterpret_cast<typename Vec2<R>::T*>(out));
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_noisy(const ProteinDev* prot, const int* chain_prot, int nchains, int nmax,
                         R* theta, R sd, unsigned long long seed, cudaStream_t st) {
  dim3 grid((nmax + 127) / 128, nchains);
  noisy_kernel<R><<<grid, 128, 0, st>>>(prot, chain_prot, theta, sd, seed);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_best(const ProteinDev* prot, const int* chain_prot, int nchains, int nmax,
                        const R* theta, R* best_theta, const double* E, double* best_E, int init,
                        cudaStream_t st) {
  (void)nmax;
  best_kernel<R><<<nchains, 128, 0, st>>>(prot, chain_prot, theta, best_theta, E, best_E, init);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_convert_in(const float* src, R* dst, long long count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  convert_in_kernel<R><<<grid_for(count, 256), 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_convert_out(const R* src, float* dst, long long count, cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  convert_out_kernel<R><<<grid_for(count, 256), 256, 0, st>>>(src, dst, count);
  return cudaGetLastError();
}

template <class R>
cudaError_t launch_exchange(const ProteinDev* prot, const int* chain_prot, int nchains, int K,
                            const double* ladder, double T_scale, int parity,
                            unsigned long long seed, unsigned long long round, R* theta,
                            double* E, long long* accepted, cudaStream_t st) {
  const int threads = 256;
  const long long total = (long long)nchains * 32;
  exchange_kernel<R><<<(int)((total + threads - 1) / threads), threads, 0, st>>>(
      prot, chain_prot, nchains, K, ladder, T_scale, parity, seed, round, theta, E, accepted);
  return cudaGetLastError();
}

cudaError_t launch_philox_fill(unsigned long long seed, unsigned chain, unsigned long long t0,
                               unsigned stream, long long count, uint4* words, float* z, float* u,
                               cudaStream_t st) {
  if (count <= 0) return cudaSuccess;
  philox_kernel<<<grid_for(count, 256), 256, 0, st>>>(seed, chain, t0, stream, count, words, z, u);
  return cudaGetLastError();
}

#define AMH_MISC_INST(R)                                                                           \
  template cudaError_t grad_set_smem<R>(size_t);                                                   \
  template cudaError_t launch_grad<R>(const ProteinDev*, int, int, const R*, int, double*, R*,     \
                                      Tab<R>, Geom<R>, cudaStream_t);                              \
  template cudaError_t launch_prep_table<R>(const double*, long long, int, int, int, R*,           \
                                            cudaStream_t);                                         \
  template cudaError_t launch_noisy<R>(const ProteinDev*, const int*, int, int, R*, R,             \
                                       unsigned long long, cudaStream_t);                          \
  template cudaError_t launch_best<R>(const ProteinDev*, const int*, int, int, const R*, R*,        \
                                      const double*, double*, int, cudaStream_t);                  \
  template cudaError_t launch_convert_in<R>(const float*, R*, long long, cudaStream_t);            \
  template cudaError_t launch_exchange<R>(const ProteinDev*, const int*, int, int, const double*,  \
                                          double, int, unsigned long long, unsigned long long, R*, \
                                          double*, long long*, cudaStream_t);                      \
  template cudaError_t launch_convert_out<R>(const R*, float*, long long, cudaStream_t);

AMH_MISC_INST(float)
AMH_MISC_INST(double)

}  // namespace amh
