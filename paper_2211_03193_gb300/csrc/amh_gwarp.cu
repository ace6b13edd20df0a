// amh_gwarp.cu -- global Metropolis sweeps (Eqs. 1-3, Alg. 1 first loop)
// by chain groups: G warps (1, 2 or 4) per chain, FP32, flat far field
// skipped.
//
// A CTA holds S chain slots of G warps each.  A slot takes chains from the
// work queue and runs a chain's proposals on its own: its warps meet at a
// named barrier of their own (a warp alone at __syncwarp), never at a
// CTA-wide one, so a slot waiting on a map, a sphere or a table fetch holds
// up no other chain.  With G = 2 the 1024 chains of the L = 300 workload
// are resident at once.
//
// Per proposal (the pair 2i-1, 2i = psi_{i-1}, phi_i shares the pivot
// p = i and is scored in one pass, as in the CTA kernel): lanes 0-2 of the
// slot's first warp form the rigid maps A1, A2 and A21 of the moving side
// (the side of the pivot with fewer residues, Sec. 2.4 step 2); the far field
// is dropped by three nested exact tests (see wblock), the surviving pairs of
// Eq. 5 are evaluated, each warp on its share of the chunk pairs, and the
// Metropolis test of Eq. 1 is taken by every thread alike from the warps'
// sums added in a fixed order.
//
// The fixed side's C-betas are cut into absolute chunks of kPairChunk atoms
// with bounding spheres that are kept across proposals: chunk j remembers
// the atom range [lo, hi) that has not moved since its sphere was computed
// (a commit of the moving side [m0, m1) removes that range), and a sphere is
// recomputed only when a proposal's fixed part of the chunk is not inside
// it.  Within a sweep the fixed side is [p, L) while p <= L/2 and [0, p)
// after, so most spheres are computed once or twice per sweep.
#include "amh_internal.h"

namespace amh {

namespace {

constexpr int kWC = kPairChunk;  // C-betas per chunk: chunk j holds atoms [kWC j, kWC j + kWC)
constexpr int kWDraw = 64;       // proposals whose draws are made ahead
constexpr size_t kKbBytes = 1792;  // residue-transform basis: 216 doubles, 128-byte rounded

__host__ __device__ inline size_t wal(size_t x) { return (x + 15) & ~size_t(15); }

constexpr int kBatch = 32;  // pairs evaluated at a time: one per lane
constexpr int kPairCap = 32 * kWC + kBatch;  // one round of 32 items of kWC pairs plus a partial batch
constexpr int kMaxG = 4;                     // warps per chain at most

// Shared memory of one chain slot (a chain of up to Lmax residues, G warps):
// the chain's state, then each warp's pair lists.
struct WLayout {
  size_t cb, fsph, msph, isph, maps, theta, bb, draws, clean, part, dpart, scan, misc;
  size_t warp0, warp_bytes, plist, kp, total;
  int nJ;
  __host__ __device__ WLayout(int Lmax, int G) {
    nJ = (Lmax + kWC - 1) / kWC;
    size_t o = 0;
    cb = o;    o = wal(o + sizeof(Pt4<float>) * (size_t)Lmax);
    fsph = o;  o = wal(o + sizeof(Pt4<float>) * (size_t)nJ);
    msph = o;  o = wal(o + sizeof(Pt4<float>) * (size_t)nJ);
    isph = o;  o = wal(o + sizeof(Pt4<float>) * (size_t)(Lmax / 2 + 1));
    maps = o;  o = wal(o + sizeof(float) * 40);
    theta = o; o = wal(o + sizeof(float) * 2 * (size_t)Lmax);
    bb = o;    o = wal(o + sizeof(float) * 9 * (size_t)Lmax);
    draws = o; o = wal(o + sizeof(float) * 2 * kWDraw);
    clean = o; o = wal(o + sizeof(int) * (size_t)nJ);
    part = o;  o = wal(o + sizeof(float) * 4 * kMaxG);
    dpart = o; o = wal(o + sizeof(double) * kMaxG);
    scan = o;  o = wal(o + sizeof(double) * 12 * kMaxG);
    misc = o;  o = wal(o + sizeof(int) * 4);
    warp0 = o;
    plist = 0;
    kp = wal(sizeof(unsigned) * kPairCap);
    warp_bytes = wal(kp + sizeof(unsigned short) * 32);
    o += (size_t)G * warp_bytes;
    total = (o + 127) & ~size_t(127);
  }
};

struct WShm {
  Pt4<float>* cb;        // [L] C-betas (x, y, z, 0)
  Pt4<float>* fsph;      // [chunk] bounding sphere of the chunk's C-betas (centre, radius)
  Pt4<float>* msph;      // [moving chunk] sphere holding its atoms' image spheres
  Pt4<float>* isph;      // [moving atom] sphere of the atom's images under the moves
  float* maps;           // A1 [0,12), A2 [12,24), A21 [24,36); thn [36,38), ln u [38,40)
  float* theta;          // [n]
  float* bb;             // [i][v][xyz]: v 0 CA_i, 1 unit N_i -> CA_i, 2 unit CA_i -> C_i
  float* draws;          // [kWDraw][2]: (z, ln u)
  int* clean;            // [chunk] lo | hi << 16: atoms unmoved since the sphere was made
  float* part;           // [warp][4] the warps' Delta-E sums
  double* dpart;         // [warp] the warps' energy sums
  double* scan;          // [warp][12] the chain build's warp totals
  int* misc;             // [0] the slot's chain (queue index), [1] best-state flag
  unsigned* plist;       // this warp's pairs within reach, (moving atom << 16 | fixed atom)
  unsigned short* kp;    // this warp's chunk pairs within reach, of one round
  __device__ WShm(unsigned char* base, const WLayout& l, int g) {
    cb = (Pt4<float>*)(base + l.cb);
    fsph = (Pt4<float>*)(base + l.fsph);
    msph = (Pt4<float>*)(base + l.msph);
    isph = (Pt4<float>*)(base + l.isph);
    maps = (float*)(base + l.maps);
    theta = (float*)(base + l.theta);
    bb = (float*)(base + l.bb);
    draws = (float*)(base + l.draws);
    clean = (int*)(base + l.clean);
    part = (float*)(base + l.part);
    dpart = (double*)(base + l.dpart);
    scan = (double*)(base + l.scan);
    misc = (int*)(base + l.misc);
    unsigned char* wb = base + l.warp0 + (size_t)g * l.warp_bytes;
    plist = (unsigned*)(wb + l.plist);
    kp = (unsigned short*)(wb + l.kp);
  }
  __device__ V3<float> x(int i) const {
    const Pt4<float> p = cb[i];
    return v3<float>(p.x, p.y, p.z);
  }
  __device__ void set_x(int i, V3<float> v) {
    Pt4<float> p;
    p.x = v.x;
    p.y = v.y;
    p.z = v.z;
    p.w = 0.f;
    cb[i] = p;
  }
  __device__ V3<float> axis(int i, int v) const {
    const float* q = bb + i * 9 + v * 3;
    return v3<float>(q[0], q[1], q[2]);
  }
  __device__ void set_axis(int i, int v, V3<float> a) {
    float* q = bb + i * 9 + v * 3;
    q[0] = a.x;
    q[1] = a.y;
    q[2] = a.z;
  }
};

// The threads of one chain slot: t in [0, nt), warp g of G, and the slot's
// meeting point (its own named barrier, or __syncwarp for one warp).
struct Grp {
  int t, nt, g, G, lane, bar;
  __device__ void sync() const {
    if (G == 1)
      __syncwarp();
    else
      asm volatile("bar.sync %0, %1;" ::"r"(bar), "r"(nt) : "memory");
  }
};

__device__ __forceinline__ float wdist2(V3<float> a, V3<float> b) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}

__device__ __forceinline__ float wsum(float v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}
__device__ __forceinline__ double wsumd(double v) {
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  return v;
}

// G(s) of the slot's chain in FP64 (a parallel scan of residue transforms
// over the slot's threads), stored in FP32; every chunk sphere becomes stale.
__device__ void wrebuild(WShm& w, const Grp& q, const Geom<double>& g, const double* kb, int L,
                         int nJ) {
  q.sync();
  build_chain_group(
      g, kb, L, q.t, q.nt, [&](int k) { return (double)w.theta[k]; },
      [&](int i, V3<double> N, V3<double> CA, V3<double> Cc, V3<double> CB) {
        w.set_axis(i, 0, v3<float>((float)CA.x, (float)CA.y, (float)CA.z));
        const V3<double> u1 = unit(CA - N), u2 = unit(Cc - CA);
        w.set_axis(i, 1, v3<float>((float)u1.x, (float)u1.y, (float)u1.z));
        w.set_axis(i, 2, v3<float>((float)u2.x, (float)u2.y, (float)u2.z));
        w.set_x(i, v3<float>((float)CB.x, (float)CB.y, (float)CB.z));
      },
      w.scan, [&]() { q.sync(); });
  for (int j = q.t; j < nJ; j += q.nt) w.clean[j] = 0;
  q.sync();
}

// Bounding spheres of the chunks that hold fixed atoms [f0, f1): a chunk
// whose fixed part lies inside its unmoved range keeps its sphere, the others
// get one over the whole chunk (box centre, largest distance).
__device__ void wspheres(WShm& w, const Grp& g, int L, int f0, int f1) {
  const int j0 = f0 / kWC, j1 = (f1 - 1) / kWC;
  for (int j = j0 + g.t; j <= j1; j += g.nt) {
    const int fa = max(kWC * j, f0), fb = min(kWC * j + kWC, f1);
    const int cl = w.clean[j];
    if ((cl & 0xffff) <= fa && fb <= (cl >> 16)) continue;
    const int ca = kWC * j, ce = min(ca + kWC, L);
    V3<float> lo = w.x(ca), hi = lo;
    for (int f = ca + 1; f < ce; ++f) {
      const V3<float> y = w.x(f);
      lo = v3<float>(fminf(lo.x, y.x), fminf(lo.y, y.y), fminf(lo.z, y.z));
      hi = v3<float>(fmaxf(hi.x, y.x), fmaxf(hi.y, y.y), fmaxf(hi.z, y.z));
    }
    const V3<float> o = (lo + hi) * 0.5f;
    float r2 = 0.f;
    for (int f = ca; f < ce; ++f) r2 = fmaxf(r2, wdist2(w.x(f), o));
    Pt4<float> s;
    s.x = o.x;
    s.y = o.y;
    s.z = o.z;
    s.w = sqrtf(r2);
    w.fsph[j] = s;
    w.clean[j] = ca | (ce << 16);
  }
  g.sync();
}

// One straddle pair (moving atom m, fixed atom f): its terms at the current
// coordinates and under the moves, added to the Delta-E sums.
template <bool FUSED, bool TEX>
__device__ __forceinline__ void wpair(const WShm& w, const Tab<float>& tb, long long tab_off, int L,
                                      int m, int f, const Move<float>& A1, const Move<float>& A2,
                                      const Move<float>& A21, float& acc1, float& acc2, float& acc21) {
  const V3<float> xm = w.x(m), xf = w.x(f);
  const int r = m < f ? row_of(L, m, f) : row_of(L, f, m);
  const V3<float> y1 = move_apply(A1, xm);
  float e0, e1, e2 = 0.f, e21 = 0.f;
  if constexpr (TEX) {
    const int rowe = (int)tab_off + r * tb.Bp;
    e0 = pair_term_tex(rowe, dist_fast(xf, xm), tb);
    e1 = pair_term_tex(rowe, dist_fast(xf, y1), tb);
    if (FUSED) {
      e2 = pair_term_tex(rowe, dist_fast(xf, move_apply(A2, xm)), tb);
      e21 = pair_term_tex(rowe, dist_fast(xf, move_apply(A21, xm)), tb);
    }
  } else {
    const float2* row = tb.E + tab_off + (long long)r * tb.Bp;
    e0 = pair_term(row, dist_fast(xf, xm), tb);
    e1 = pair_term(row, dist_fast(xf, y1), tb);
    if (FUSED) {
      e2 = pair_term(row, dist_fast(xf, move_apply(A2, xm)), tb);
      e21 = pair_term(row, dist_fast(xf, move_apply(A21, xm)), tb);
    }
  }
  acc1 += e1 - e0;
  if (FUSED) {
    acc2 += e2 - e0;
    acc21 += e21 - e1;
  }
}

__device__ __forceinline__ V3<float> wc(Pt4<float> p) { return v3<float>(p.x, p.y, p.z); }

// Delta-E of move 1, of move 2 and of move 2 after move 1 (FUSED) over the
// straddle block without its flat far field; every lane returns the sums.
// A straddle pair adds zero when all its distances, before and after the
// moves, lie beyond the last bin centre; three nested tests, each exact for
// the pairs it drops, find the others: (1) each moving atom's images (the
// atom and its places under the moves) get a sphere, and each chunk of
// moving atoms a sphere holding those; (2) a chunk pair (moving chunk,
// fixed chunk) is dropped when their spheres stay `cut` apart; (3) for the
// kept chunk pairs, a moving atom is dropped against a fixed chunk, and
// then a pair against its fixed atom, by the same reach.  The pairs left
// are listed and evaluated 32 at a time, every lane on one pair.
template <bool FUSED, bool TEX>
__device__ void wblock(WShm& w, const Grp& grp, const Tab<float>& tb, long long tab_off, int L,
                       int m0, int m1, int f0, int f1, float cut, float& s1, float& s2,
                       float& s21, unsigned long long& count) {
  const int lane = grp.lane;
  Move<float> A1, A2, A21;
  load_rot(w.maps, A1);
  A2 = A1;
  A21 = A1;
  if (FUSED) {
    load_rot(w.maps + 12, A2);
    load_move21(w.maps + 24, A1.p, A21);
  }
  const int nM = m1 - m0;
  // (1) image spheres of the moving atoms
  for (int mi = grp.t; mi < nM; mi += grp.nt) {
    const V3<float> xm = w.x(m0 + mi);
    const V3<float> y1 = move_apply(A1, xm);
    V3<float> o;
    float r2;
    if (FUSED) {
      const V3<float> y2 = move_apply(A2, xm), y21 = move_apply(A21, xm);
      o = (xm + y1 + y2 + y21) * 0.25f;
      r2 = fmaxf(fmaxf(wdist2(xm, o), wdist2(y1, o)), fmaxf(wdist2(y2, o), wdist2(y21, o)));
    } else {
      o = (xm + y1) * 0.5f;
      r2 = fmaxf(wdist2(xm, o), wdist2(y1, o));
    }
    Pt4<float> q;
    q.x = o.x;
    q.y = o.y;
    q.z = o.z;
    q.w = sqrtf(r2);
    w.isph[mi] = q;
  }
  grp.sync();
  // ... and of the moving chunks: centred on a middle atom's image sphere,
  // reaching every image sphere of the chunk
  const int jm0 = m0 / kWC, nJm = (m1 - 1) / kWC - jm0 + 1;
  const int jf0 = f0 / kWC, nJf = (f1 - 1) / kWC - jf0 + 1;
  for (int jj = grp.t; jj < nJm; jj += grp.nt) {
    const int a0 = max(kWC * (jm0 + jj), m0) - m0, a1 = min(kWC * (jm0 + jj) + kWC, m1) - m0;
    const V3<float> c = wc(w.isph[(a0 + a1 - 1) >> 1]);
    float R = 0.f;
    for (int q = a0; q < a1; ++q) {
      const Pt4<float> t = w.isph[q];
      R = fmaxf(R, sqrtf(wdist2(wc(t), c)) + t.w);
    }
    Pt4<float> q;
    q.x = c.x;
    q.y = c.y;
    q.z = c.z;
    q.w = R;
    w.msph[jj] = q;
  }
  grp.sync();
  // (2)-(3) each warp takes every G-th round of 32 chunk pairs, with its own
  // lists
  float acc1 = 0.f, acc2 = 0.f, acc21 = 0.f;
  unsigned long long npairs = 0;
  int np = 0;  // pairs listed and not yet evaluated (the same on every lane)
  const int ncp = nJm * nJf;
  for (int cp0 = 32 * grp.g; cp0 < ncp; cp0 += 32 * grp.G) {
    // (2) 32 chunk pairs
    const int cp = cp0 + lane;
    bool keep = false;
    if (cp < ncp) {
      const int jm = cp / nJf, jf = cp - jm * nJf;
      const Pt4<float> a = w.msph[jm], b = w.fsph[jf0 + jf];
      const float lim = a.w + b.w + cut;
      keep = wdist2(wc(a), wc(b)) < lim * lim;
    }
    const unsigned kb = __ballot_sync(0xffffffffu, keep);
    if (!kb) continue;
    if (keep) w.kp[__popc(kb & ((1u << lane) - 1u))] = (unsigned short)cp;
    __syncwarp();
    const int nit = __popc(kb) * kWC;
    // (3) their (moving atom, fixed chunk) items, 32 at a time
    for (int it0 = 0; it0 < nit; it0 += 32) {
      const int it = it0 + lane;
      unsigned mask = 0;
      int m = 0, fb = 0;
      if (it < nit) {
        const int cpk = w.kp[it / kWC];
        const int jm = cpk / nJf, J = jf0 + (cpk - jm * nJf);
        m = kWC * (jm0 + jm) + it % kWC;
        if (m >= m0 && m < m1) {
          const Pt4<float> t = w.isph[m - m0], b = w.fsph[J];
          const float reach = t.w + cut, lim = reach + b.w;
          const V3<float> o = wc(t);
          if (wdist2(o, wc(b)) < lim * lim) {
            fb = max(kWC * J, f0);
            const int fe = min(kWC * J + kWC, f1);
            const float r2 = reach * reach;
            for (int f = fb; f < fe; ++f)
              if (wdist2(w.x(f), o) < r2) mask |= 1u << (f - fb);
          }
        }
      }
      const int cnt = __popc(mask);
      int incl = cnt;
#pragma unroll
      for (int off = 1; off < 32; off <<= 1) {
        const int v = __shfl_up_sync(0xffffffffu, incl, off);
        if (lane >= off) incl += v;
      }
      const int total = __shfl_sync(0xffffffffu, incl, 31);
      int pos = np + incl - cnt;
      while (mask) {
        const int q = __ffs(mask) - 1;
        mask &= mask - 1;
        w.plist[pos++] = ((unsigned)m << 16) | (unsigned)(fb + q);
      }
      np += total;
      __syncwarp();
      if (np >= kBatch) {
        // evaluate whole batches; the rest waits
        const int nrun = np - np % kBatch;
        for (int q = lane; q < nrun; q += 32) {
          const unsigned e = w.plist[q];
          wpair<FUSED, TEX>(w, tb, tab_off, L, (int)(e >> 16), (int)(e & 0xffffu), A1, A2, A21,
                            acc1, acc2, acc21);
        }
        npairs += (unsigned long long)(nrun >> 5);
        // move the rest (< kBatch pairs) to the front: read all, then write
        const int rem = np - nrun;
        unsigned v[kBatch / 32];
#pragma unroll
        for (int r = 0; r < kBatch / 32; ++r)
          v[r] = lane + 32 * r < rem ? w.plist[nrun + lane + 32 * r] : 0u;
        __syncwarp();
#pragma unroll
        for (int r = 0; r < kBatch / 32; ++r)
          if (lane + 32 * r < rem) w.plist[lane + 32 * r] = v[r];
        __syncwarp();
        np = rem;
      }
    }
  }
  for (int q = lane; q < np; q += 32) {
    const unsigned e = w.plist[q];
    wpair<FUSED, TEX>(w, tb, tab_off, L, (int)(e >> 16), (int)(e & 0xffffu), A1, A2, A21, acc1,
                      acc2, acc21);
    npairs += 1;
  }
  count += npairs * (FUSED ? 4 : 2);
  acc1 = wsum(acc1);
  acc2 = wsum(acc2);
  acc21 = wsum(acc21);
  if (grp.G == 1) {
    s1 = acc1;
    s2 = acc2;
    s21 = acc21;
    return;
  }
  // the warps' sums, added in warp order by every thread
  if (lane == 0) {
    w.part[4 * grp.g] = acc1;
    w.part[4 * grp.g + 1] = acc2;
    w.part[4 * grp.g + 2] = acc21;
  }
  grp.sync();
  s1 = s2 = s21 = 0.f;
  for (int h = 0; h < grp.G; ++h) {
    s1 += w.part[4 * h];
    s2 += w.part[4 * h + 1];
    s21 += w.part[4 * h + 2];
  }
  grp.sync();
}

// V of the slot's chain from its current coordinates: FP32 terms, FP64 sums
// (Eq. 5 over a < b); every thread returns it.
__device__ double wenergy(const WShm& w, const Grp& g, const Tab<float>& tb, long long tab_off,
                          int L) {
  const int nch = (L - 1 + kWC - 1) / kWC;
  const int items = L * nch;
  double acc = 0.0;
  for (int it = g.t; it < items; it += g.nt) {
    const int a = it / nch, ch = it - a * nch;
    const int b0 = a + 1 + ch * kWC;
    const int b1 = min(L, b0 + kWC);
    if (b0 >= b1) continue;
    const V3<float> xa = w.x(a);
    const float2* row = tb.E + tab_off + (long long)row_of(L, a, b0) * tb.Bp;
    float part = 0.f;
    for (int b = b0; b < b1; ++b, row += tb.Bp) part += pair_term(row, dist_(xa, w.x(b)), tb);
    acc += (double)part;
  }
  acc = wsumd(acc);
  if (g.G == 1) return acc;
  if (g.lane == 0) w.dpart[g.g] = acc;
  g.sync();
  double e = 0.0;
  for (int h = 0; h < g.G; ++h) e += w.dpart[h];
  g.sync();
  return e;
}

template <bool TEX>
__device__ void wrun_chain(WShm& w, const Grp& q, const SweepArgs<float>& a, const double* kb,
                           const GroupDev& G, const ProteinDev& P, int nJ) {
  const int t = q.t, nt = q.nt;
  const int L = P.L, n = P.n;
  const int chain = G.chain0;
  const long long toff = P.tors0 + (long long)(chain - P.chain0) * n;
  for (int k = t; k < n; k += nt) w.theta[k] = a.theta[toff + k];
  const long long t0 = a.tcount[chain];
  const long long steps = a.steps_are_sweeps ? a.steps * n : a.steps;
  const double lad = a.ladder ? a.ladder[(chain - P.chain0) % a.ladder_K] : 1.0;
  long long sw = 0;  // sweep of the call (scheduled calls start on a sweep boundary)
  // decisions in FP32, the form's precision (the product's rounding is far
  // inside the 1e-5 tie margin; the FP64 pipe runs at 1/64 of the FP32 rate)
  float Tf = (float)(a.T_of(0) * lad);
  float sig = a.sigma_of(0);
  const bool traced = chain < a.trace_chains;
  // decisions need Delta-E only and the exit recomputes V from scratch, so
  // the entry and periodic resyncs rebuild the coordinates alone
  wrebuild(w, q, a.geom64, kb, L, nJ);
  long long since = 0, nacc = 0;
  unsigned long long count = 0;
  long long d0 = 0, dend = 0;
  int kn = (int)(t0 % n);
  for (long long j = 0; j < steps;) {
    if (j + 2 > dend) {
      q.sync();
      d0 = j;
      dend = j + kWDraw;
      for (int r = t; r < kWDraw; r += nt) {
        float z, lnu;
        normal_and_lnu(draw_words(a.seed, (uint32_t)chain, (unsigned long long)(t0 + j + r), 0u),
                       &z, &lnu);
        w.draws[2 * r] = z;
        w.draws[2 * r + 1] = lnu;
      }
      q.sync();
    }
    const long long tp = t0 + j;
    const int k = kn;
    if (k == 0 && j > 0 && a.nsched) {
      ++sw;
      Tf = (float)(a.T_of(sw) * lad);
      sig = a.sigma_of(sw);
    }
    if (since >= a.resync_every || (k == 0 && j > 0)) {
      wrebuild(w, q, a.geom64, kb, L, nJ);
      since = 0;
    }
    const bool fused = (k & 1) && (k + 1 < n) && (j + 1 < steps);
    const int p = (k + 1) >> 1;
    const bool up = p <= L - p;  // move the upstream side (it is the smaller)
    const int m0 = up ? 0 : p, m1 = up ? p : L;
    const int f0 = up ? p : 0, f1 = up ? L : p;
    const bool dead = (k == 0) || (k == n - 1);
    // three lanes form the maps: lane 0 move 1's A1, lane 1 move 2's A2
    // about its own axis, lane 2 A1 again and then move 2 about its axis as
    // move 1 left it, composed after A1 (the CTA kernel's arithmetic)
    if (t == 0 || (t < 3 && fused)) {
      const int k1 = t == 1 ? k + 1 : k;
      const float z = w.draws[2 * (j + (k1 - k) - d0)];
      const float lnu = w.draws[2 * (j + (k1 - k) - d0) + 1];
      const float th = w.theta[k1];
      const float thn = propose(th, z, sig, a.lattice_K);
      if (t < 2) {
        w.maps[36 + t] = thn;
        w.maps[38 + t] = lnu;
      }
      if (!dead) {
        // k1 odd: psi_i about CA_i -> C_i; k1 even: phi_i about N_i -> CA_i
        const int i = k1 >> 1;
        const float d = wrap_angle(thn - th);
        const Move<float> A = move_rotation(w.axis(i, 0), w.axis(i, (k1 & 1) ? 2 : 1), up ? -d : d);
        if (t < 2) {
          store_move(w.maps + 12 * t, A, A.p);
        } else {
          const float z2 = w.draws[2 * (j + 1 - d0)];
          const float th2 = w.theta[k + 1];
          const float d2 = wrap_angle(propose(th2, z2, sig, a.lattice_K) - th2);
          const V3<float> P2 = w.axis(p, 0), u2 = w.axis(p, 1);  // phi_p: N_p -> CA_p
          const V3<float> P2m = up ? P2 : move_apply(A, P2);
          const V3<float> u2m = up ? u2 : move_lin(A, u2);
          const Move<float> A21 = move_compose(move_rotation(P2m, u2m, up ? -d2 : d2), A);
          store_move(w.maps + 24, A21, A21.q);
        }
      }
    }
    q.sync();
    if (dead) {
      // phi_0 and psi_{L-1} move no C-beta: Delta-E = 0, always accepted
      const float thn = w.maps[36], lnu = w.maps[38];
      const int acc = lnu * Tf < -0.f;
      if (t == 0) {
        if (acc) w.theta[k] = thn;
        if (traced && tp < a.trace_cap) {
          TraceRec r;
          r.k = k;
          r.accept = acc;
          r.theta_new = (double)thn;
          r.lnu = (double)lnu;
          r.dE = 0.0;
          a.trace[(size_t)chain * a.trace_cap + tp] = r;
        }
      }
      nacc += acc;
      q.sync();
      j += 1;
      since += 1;
      kn = k + 1 < n ? k + 1 : 0;
      continue;
    }
    wspheres(w, q, L, f0, f1);
    float s1, s2, s21;
    if (fused)
      wblock<true, TEX>(w, q, a.tab, P.tab_off, L, m0, m1, f0, f1, a.far_cut, s1, s2, s21, count);
    else
      wblock<false, TEX>(w, q, a.tab, P.tab_off, L, m0, m1, f0, f1, a.far_cut, s1, s2, s21,
                         count);
    // Eq. 1 with T > 0: ln u < -dE / T  <=>  T ln u < -dE, taken by every thread
    const float thn1 = w.maps[36], lnu1 = w.maps[38];
    const int acc1 = lnu1 * Tf < -s1;
    int code = acc1, acc2 = 0;
    float e2 = 0.f;
    if (fused) {
      e2 = acc1 ? s21 : s2;
      acc2 = w.maps[39] * Tf < -e2;
      if (acc2) code = acc1 ? 3 : 2;
    }
    if (t == 0) {
      if (acc1) w.theta[k] = thn1;
      if (traced && tp < a.trace_cap) {
        TraceRec r;
        r.k = k;
        r.accept = acc1;
        r.theta_new = (double)thn1;
        r.lnu = (double)lnu1;
        r.dE = (double)s1;
        a.trace[(size_t)chain * a.trace_cap + tp] = r;
      }
      if (fused) {
        if (acc2) w.theta[k + 1] = w.maps[37];
        if (traced && tp + 1 < a.trace_cap) {
          TraceRec r;
          r.k = k + 1;
          r.accept = acc2;
          r.theta_new = (double)w.maps[37];
          r.lnu = (double)w.maps[39];
          r.dE = (double)e2;
          a.trace[(size_t)chain * a.trace_cap + tp + 1] = r;
        }
      }
    }
    nacc += acc1 + acc2;
    if (code) {
      // commit: the moving side turns by the accepted map; an upstream move
      // turns only C-betas (the rest of this sweep rotates about bonds at or
      // after the pivot, and a new sweep starts from a rebuild)
      Move<float> A;
      if (code < 3)
        load_rot(w.maps + 12 * (code - 1), A);
      else
        load_move21(w.maps + 24, w.maps + 9, A);
      const int per = up ? 1 : 4;
      const int total = (m1 - m0) * per;
      for (int idx = t; idx < total; idx += nt) {
        const int v = up ? 3 : (idx & 3), i = m0 + (up ? idx : idx >> 2);
        if (v == 0)
          w.set_axis(i, 0, move_apply(A, w.axis(i, 0)));
        else if (v < 3)
          w.set_axis(i, v, move_lin(A, w.axis(i, v)));
        else
          w.set_x(i, move_apply(A, w.x(i)));
      }
      // the chunks' unmoved ranges lose [m0, m1)
      if (up) {
        for (int jj = t; jj <= (p - 1) / kWC; jj += nt) {
          const int cl = w.clean[jj];
          w.clean[jj] = max(cl & 0xffff, p) | (cl & ~0xffff);
        }
      } else {
        for (int jj = p / kWC + t; jj < nJ; jj += nt) {
          const int cl = w.clean[jj];
          w.clean[jj] = (cl & 0xffff) | (min(cl >> 16, p) << 16);
        }
      }
    }
    q.sync();
    j += fused ? 2 : 1;
    kn = k + (fused ? 2 : 1);
    if (kn >= n) kn -= n;
    since += fused ? 2 : 1;
  }
  // exit: V from scratch (FP64 sum) of the current coordinates (their drift
  // since the last rebuild is ~1e-5 A)
  q.sync();
  const double e = wenergy(w, q, a.tab, P.tab_off, L);
  if (t == 0) {
    int better = 0;
    if (!(e == e)) atomicOr(a.err, 1);  // NaN energy
    a.E_cur[chain] = e;
    a.tcount[chain] = t0 + steps;
    if (a.acc_out) a.acc_out[chain] = nacc;
    if (a.trace_count && traced)
      a.trace_count[chain] = t0 + steps < a.trace_cap ? t0 + steps : a.trace_cap;
    if (e < a.best_E[chain]) {
      a.best_E[chain] = e;
      better = 1;
    }
    w.misc[1] = better;
  }
  q.sync();
  const int better = w.misc[1];
  for (int k = t; k < n; k += nt) {
    const float v = w.theta[k];
    a.theta[toff + k] = v;
    if (better) a.best_theta[toff + k] = v;
  }
  if (a.coords) {
    const long long off = 3 * (toff / 2);
    for (int i = t; i < L; i += nt) {
      const V3<float> x = w.x(i);
      a.coords[off + 3 * i] = x.x;
      a.coords[off + 3 * i + 1] = x.y;
      a.coords[off + 3 * i + 2] = x.z;
    }
  }
  unsigned long long c = count;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) c += __shfl_xor_sync(0xffffffffu, c, off);
  if (q.lane == 0 && a.pair_count && c) {  // every pair it forms is read
    atomicAdd(a.pair_count, c);
    atomicAdd(a.pair_count + 1, c);
  }
  q.sync();
}

template <bool TEX>
__global__ void __launch_bounds__(256) gwarp_kernel(SweepArgs<float> a, int G) {
  extern __shared__ __align__(128) unsigned char smem[];
  double* kb = reinterpret_cast<double*>(smem);
  residue_basis(a.geom64, kb);  // the whole CTA, once
  const WLayout lay(a.Lmax, G);
  const int warp = threadIdx.x >> 5;
  Grp q;
  q.G = G;
  q.nt = 32 * G;
  q.g = warp % G;
  q.lane = threadIdx.x & 31;
  q.t = threadIdx.x % q.nt;
  q.bar = 1 + warp / G;  // named barrier of the slot (0 is __syncthreads)
  unsigned char* base = smem + kKbBytes + (size_t)(warp / G) * lay.total;
  WShm w(base, lay, q.g);
  for (;;) {
    if (q.t == 0) w.misc[0] = atomicAdd(a.queue, 1);
    q.sync();
    const int g = w.misc[0];
    q.sync();
    if (g >= a.ngroups) break;
    const GroupDev Gd = a.groups[g];
    wrun_chain<TEX>(w, q, a, kb, Gd, a.prot[Gd.protein], lay.nJ);
  }
}

}  // namespace

size_t gwarp_smem_bytes(int Lmax, int slots, int G) {
  return kKbBytes + (size_t)slots * WLayout(Lmax, G).total;
}

cudaError_t gwarp_set_smem(size_t optin) {
  cudaError_t e = allow_dynamic_smem(gwarp_kernel<true>, optin);
  if (e != cudaSuccess) return e;
  return allow_dynamic_smem(gwarp_kernel<false>, optin);
}

cudaError_t gwarp_occupancy(int slots, int G, size_t smem, int* per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, gwarp_kernel<true>,
                                                       32 * G * slots, smem);
}

cudaError_t launch_gwarp(const SweepArgs<float>& a, int slots, int G, int grid, cudaStream_t st) {
  const size_t sm = gwarp_smem_bytes(a.Lmax, slots, G);
  if (a.tab.tex)
    gwarp_kernel<true><<<grid, 32 * G * slots, sm, st>>>(a, G);
  else
    gwarp_kernel<false><<<grid, 32 * G * slots, sm, st>>>(a, G);
  return cudaGetLastError();
}

}  // namespace amh
