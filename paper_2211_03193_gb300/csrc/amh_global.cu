// amh_global.cu -- global Metropolis sweeps and full-energy resync.
//
// One CTA runs a group of C chains of one protein in lock-step: they share
// the torsion index k of every proposal (Alg. 1: k = 1..length(s) in
// order), so the straddle block of pairs a < p(k) <= b (the only pairs
// whose distance changes, Sec. 2.4 steps 2-3) reads the same distogram rows
// for all C chains; lanes of a warp are (chain, slice) so one row fetch is
// coalesced across the chains.  The proposal pair (2i-1, 2i) = (psi_{i-1},
// phi_i) shares the pivot p = i, so both proposals are scored in one pass:
// e(x), e(A1 x), e(A2 x) and e(A21 x) per pair give Delta-E of move 1 and
// of move 2 after either outcome of move 1, exactly as in sequential
// order.  The moving side of a proposal is the smaller one (energy is
// invariant under rigid motion).  In FP32, pairs that stay beyond the last
// bin centre are dropped by whole chunks before any distance is formed, and
// a pair whose images all lie at or past it reads no table entry (it adds
// exactly zero).  The proposals of the rest of a sweep, with the sines and
// cosines of their rotations, are made ahead by all threads.  No running
// energy is kept (a decision needs Delta-E only): the coordinates are
// rebuilt from the torsions in FP64 at entry, every resync_every proposals
// and at each new sweep, and V is recomputed from scratch (FP64 sum) when
// the call ends.
#include "amh_internal.h"

namespace amh {

namespace {

constexpr int kFC = kPairChunk;  // fixed-side atoms per work item
constexpr int kDraw = 64;          // proposals made ahead, all at once

template <class R>
struct AccT {
  using T = float;
};
template <>
struct AccT<double> {
  using T = double;
};

// Regions are 32-byte aligned so 4-wide points of either precision load
// with vector instructions.
__host__ __device__ inline size_t align16(size_t x) { return (x + 31) & ~size_t(31); }


// Dynamic shared memory layout of a global-sweep CTA.
template <class R, int C>
struct Layout {
  size_t theta, bb, cb, draws, kb, maps, list, fsph, bits, part, partf, ecur, thn, lnu, acc, commit, flag, scan,
      bars, ring, total;
  int ls;  // stride between chains of the C-beta array (odd: conflict-free 16-byte loads)
  int nm;  // moving atoms at most: stride of the chunk bits per chain
  // D ring slots per warp of 32/C rows of RB bytes (D = 0: no staging).  The
  // FP32 unstaged kernel also holds the far-field pruning's arrays: the kept
  // items, spheres of the fixed side's chunks, and per (chain, moving atom)
  // the chunks within reach as bits.
  __host__ __device__ Layout(int Lmax, int nmax, int W, int D = 0, int RB = 0) {
    const bool far = sizeof(R) == 4 && D == 0;
    const int nM = (Lmax + 1) / 2, nJ = (Lmax + kFC - 1) / kFC;
    nm = nM;
    size_t o = 0;
    theta = o; o = align16(o + sizeof(R) * (size_t)nmax * C);
    bb = o;    o = align16(o + sizeof(R) * (size_t)Lmax * 9 * C);
    ls = Lmax | 1;
    cb = o;    o = align16(o + sizeof(Pt4<R>) * (size_t)ls * C);
    draws = o; o = align16(o + sizeof(R) * 4 * kDraw * C);
    kb = o;    o = align16(o + sizeof(double) * 216);
    maps = o;  o = align16(o + sizeof(R) * 36 * C);
    list = o;  o = align16(o + (far ? sizeof(unsigned short) * (size_t)nM * nJ : 0));
    fsph = o;  o = align16(o + (far ? sizeof(Pt4<R>) * (size_t)nJ * C : 0));
    bits = o;  o = align16(o + (far ? sizeof(ChunkBits) * (size_t)nM * C : 0));
    part = o;  o = align16(o + sizeof(double) * 3 * (size_t)W * C);
    partf = o; o = align16(o + sizeof(float) * 3 * (size_t)W * C);
    ecur = o;  o = align16(o + sizeof(double) * C);
    thn = o;   o = align16(o + sizeof(R) * 2 * C);
    lnu = o;   o = align16(o + sizeof(R) * 2 * C);
    acc = o;   o = align16(o + sizeof(long long) * C);
    commit = o; o = align16(o + sizeof(int) * C);
    flag = o;  o = align16(o + sizeof(int) * C);
    scan = o;  o = align16(o + sizeof(double) * 12 * (size_t)W);
    bars = o;  o = align16(o + sizeof(unsigned long long) * (size_t)W * D);
    o = (o + 127) & ~size_t(127);
    ring = o;  o = align16(o + (size_t)W * D * (32 / C) * RB);
    total = o;
  }
};

template <class R, int C>
struct Shm {
  R* theta;  // [k][C]
  R* bb;     // [((i*3+v)*3+xyz)][C]: v 0 CA_i, 1 unit N_i -> CA_i, 2 unit CA_i -> C_i
  Pt4<R>* cb4;  // [C][ls]: chain-major, odd stride
  R* draws;     // [kDraw][C][4]: (theta', ln u, sin, cos of the rotation) of the next proposals
  double* kb;   // residue-transform basis (residue_basis), 216 doubles
  R* maps;   // [C][36]: moves A1, A2, A21 (see load_rot)
  unsigned short* list;  // items kept by the far-field test, in order
  Pt4<R>* fsph;    // [chunk][C]: centre and radius of a fixed-side chunk's C-betas
  ChunkBits* bits;  // [C][moving atom]: chunks whose pairs may not be flat
  int ls, nm;
  double* part;  // [W][C][3]: FP64 partial sums (energies; FP64 Delta-E)
  float* partf;  // [W][C][3]: FP32 partial sums of Delta-E
  double* ecur;  // [C]
  R* thn;        // [2][C]
  R* lnu;        // [2][C]
  long long* acc;
  int* commit;
  int* flag;
  double* scan;              // [W][12] warp totals of the chain-building scan
  unsigned long long* bars;  // [W][D] mbarriers of the staging rings
  unsigned char* ring;       // [W][D][32/C][RB] staged table rows
  __device__ Shm(unsigned char* base, const Layout<R, C>& l) {
    theta = (R*)(base + l.theta);
    bb = (R*)(base + l.bb);
    cb4 = (Pt4<R>*)(base + l.cb);
    draws = (R*)(base + l.draws);
    kb = (double*)(base + l.kb);
    maps = (R*)(base + l.maps);
    list = (unsigned short*)(base + l.list);
    fsph = (Pt4<R>*)(base + l.fsph);
    bits = (ChunkBits*)(base + l.bits);
    ls = l.ls;
    nm = l.nm;
    part = (double*)(base + l.part);
    partf = (float*)(base + l.partf);
    ecur = (double*)(base + l.ecur);
    thn = (R*)(base + l.thn);
    lnu = (R*)(base + l.lnu);
    acc = (long long*)(base + l.acc);
    commit = (int*)(base + l.commit);
    flag = (int*)(base + l.flag);
    scan = (double*)(base + l.scan);
    bars = (unsigned long long*)(base + l.bars);
    ring = base + l.ring;
  }
  __device__ V3<R> cb(int i, int c) const {
    const Pt4<R> p = cb4[c * ls + i];
    return v3<R>(p.x, p.y, p.z);
  }
  __device__ void set_cb(int i, int c, V3<R> v) {
    Pt4<R> p;
    p.x = v.x;
    p.y = v.y;
    p.z = v.z;
    p.w = (R)0;
    cb4[c * ls + i] = p;
  }
  // the torsion axes of residue i: both pass through CA_i; phi_i runs
  // along N_i -> CA_i, psi_i along CA_i -> C_i
  __device__ V3<R> bbv(int i, int v, int c) const {
    const R* p = bb + (size_t)((i * 3 + v) * 3) * C + c;
    return v3<R>(p[0], p[C], p[2 * C]);
  }
  __device__ void set_bbv(int i, int v, int c, V3<R> x) {
    R* p = bb + (size_t)((i * 3 + v) * 3) * C + c;
    p[0] = x.x;
    p[C] = x.y;
    p[2 * C] = x.z;
  }
};

template <class R>
__device__ __forceinline__ V3<R> to_r(V3<double> v) {
  return v3<R>((R)v.x, (R)v.y, (R)v.z);
}

// G(s) of all C chain slots, built in FP64 by all threads (a parallel scan
// of residue transforms) and stored in R: rounding the torsions' sines and
// cosines in single precision would random-walk the frame along the chain
// (~1e-4 A at L=300).  The torsion axes are kept as CA and two unit bond
// directions formed in FP64: a direction from two FP32 atoms 1.46 A apart
// would be off by up to ulp(|x|) / 1.46 A (2.6e-6 rad at 50 A), and a move
// would carry its whole side off by that angle times the move's angle.  Not
// inlined: the FP64 scan needs far more registers than the proposal loop,
// and as a call of its own it no longer sets the whole kernel's allocation
// (it runs once per sweep; its spills stay inside it).  cache (global
// memory, C * L * 12 doubles, or null): the first pass's residue
// transforms, read back by the second instead of formed again.
template <class R, int C>
__device__ __noinline__ void build_chains(Shm<R, C>& s, const Geom<double>& g, int L,
                                          double* cache) {
  build_chains_scan(
      g, s.kb, L, C, [&](int c, int k) { return (double)s.theta[k * C + c]; },
      [&](int c, int i, V3<double> N, V3<double> CA, V3<double> Cc, V3<double> CB) {
        s.set_bbv(i, 0, c, to_r<R>(CA));
        s.set_bbv(i, 1, c, to_r<R>(unit(CA - N)));
        s.set_bbv(i, 2, c, to_r<R>(unit(Cc - CA)));
        s.set_cb(i, c, to_r<R>(CB));
      },
      s.scan, cache);
}

// Reduce three per-lane partial sums over the slices of each chain and
// over warps; results land in s.part[0..W) and the caller sums them.
template <class R, int C>
__device__ __forceinline__ void reduce3(Shm<R, C>& s, double a0, double a1, double a2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = C; off < 32; off <<= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, off);
    a1 += __shfl_xor_sync(0xffffffffu, a1, off);
    a2 += __shfl_xor_sync(0xffffffffu, a2, off);
  }
  if (lane < C) {
    double* p = s.part + (size_t)(warp * C + lane) * 3;
    p[0] = a0;
    p[1] = a1;
    p[2] = a2;
  }
}

// The same for the straddle blocks' partial sums, in FP32 (each partial is
// an FP32 sum already; the FP64 pipe is the scarce one): results in s.partf.
template <class R, int C>
__device__ __forceinline__ void reduce3f(Shm<R, C>& s, float a0, float a1, float a2) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int off = C; off < 32; off <<= 1) {
    a0 += __shfl_xor_sync(0xffffffffu, a0, off);
    a1 += __shfl_xor_sync(0xffffffffu, a1, off);
    a2 += __shfl_xor_sync(0xffffffffu, a2, off);
  }
  if (lane < C) {
    float* p = s.partf + (size_t)(warp * C + lane) * 3;
    p[0] = a0;
    p[1] = a1;
    p[2] = a2;
  }
}

// Full energy of every chain slot from the current coordinates: FP32 (or
// FP64) pair terms, FP64 sums (Eq. 5 over a<b).  Ends with s.ecur set.
template <class R, int C>
__device__ void full_energy(Shm<R, C>& s, const Tab<R>& tb, long long tab_off, int L) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  constexpr int S = 32 / C;
  const int c = lane % C, sl = lane / C;
  const int gs = warp * S + sl, G = W * S;
  const int nch = (L - 1 + kFC - 1) / kFC;
  const int items = L * nch;
  double acc = 0.0;
  for (int it = gs; it < items; it += G) {
    const int a = it / nch, ch = it - a * nch;
    const int b0 = a + 1 + ch * kFC;
    const int b1 = min(L, b0 + kFC);
    if (b0 >= b1) continue;
    const V3<R> xa = s.cb(a, c);
    const auto* row = tb.E + tab_off + (long long)row_of(L, a, b0) * tb.Bp;
    typename AccT<R>::T part = 0;
    for (int b = b0; b < b1; ++b, row += tb.Bp) part += pair_term(row, dist_(xa, s.cb(b, c)), tb);
    acc += (double)part;
  }
  reduce3(s, acc, 0.0, 0.0);
  __syncthreads();
  if (threadIdx.x < C) {
    double e = 0.0;
    for (int w = 0; w < W; ++w) e += s.part[(size_t)(w * C + threadIdx.x) * 3];
    s.ecur[threadIdx.x] = e;
  }
  __syncthreads();
}

// Coordinates from the torsions in FP64 (G(s) of Sec. 2.1), rounded to R.
template <class R, int C>
__device__ void rebuild(Shm<R, C>& s, const SweepArgs<R>& a, const ProteinDev& P) {
  __syncthreads();
  build_chains(s, a.geom64, P.L,
               a.tcache ? a.tcache + (size_t)blockIdx.x * C * a.Lmax * 12 : nullptr);
  __syncthreads();
}

template <class R, int C>
__device__ void resync(Shm<R, C>& s, const SweepArgs<R>& a, const ProteinDev& P) {
  rebuild(s, a, P);
  full_energy(s, a.tab, P.tab_off, P.L);
}

// Straddle-block Delta-E (moving side [m0, m1), fixed side [f0, f1)).
// Items are (moving atom, chunk of kFC fixed atoms); with LIST the items
// run are the nlist entries of `list` (item indices mi * nch + ch).  FP32:
// a pair whose images all lie at or past the last bin centre adds exactly
// zero (each reads the row's one flat entry), so its entries are not read;
// nread counts the terms read (4 per pair of a fused proposal pair, 2
// otherwise), for the chain slots set in `real`.
template <class R, int C, bool FUSED, bool TEX, bool LIST = false>
__device__ void pair_block(Shm<R, C>& s, const Tab<R>& tb, long long tab_off, int L, int m0,
                           int m1, int f0, int f1, unsigned real, unsigned& nread,
                           const unsigned short* list = nullptr, int nlist = 0) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  constexpr int S = 32 / C;
  const int c = lane % C, sl = lane / C;
  const int gs = warp * S + sl, G = W * S;
  const int nF = f1 - f0;
  const int nch = (nF + kFC - 1) / kFC;
  const int items = LIST ? nlist : (m1 - m0) * nch;
  const unsigned live = (real >> c) & 1u;
  typename AccT<R>::T acc1 = 0, acc2 = 0, acc21 = 0;
  for (int q = gs; q < items; q += G) {
    const int it = LIST ? (int)list[q] : q;
    const int mi = it / nch, ch = it - mi * nch;
    const int m = m0 + mi;
    const V3<R> xm = s.cb(m, c);
    // the maps are read per item (only the moved positions stay live in the
    // pair loop, leaving registers for more loads in flight)
    Move<R> A;
    load_rot(s.maps + 36 * c, A);
    const V3<R> y1 = move_apply(A, xm);
    V3<R> y2, y21;
    if (FUSED) {
      load_move21(s.maps + 36 * c + 24, A.p, A);
      y21 = move_apply(A, xm);
      load_rot(s.maps + 36 * c + 12, A);
      y2 = move_apply(A, xm);
    }
    const int fb = f0 + ch * kFC, fe = min(fb + kFC, f1);
    // rows of the pairs (f, m): contiguous in f when m < f; when f < m,
    // r(f+1, m) - r(f, m) = L - f - 2
    const bool mfirst = m < fb;
    const int r0 = mfirst ? row_of(L, m, fb) : row_of(L, fb, m);
    const auto* row = tb.E + tab_off + (long long)r0 * tb.Bp;
    int rowe = (int)tab_off + r0 * tb.Bp;  // entry index (texture path)
    int step = mfirst ? 1 : L - fb - 2;
    const int dstep = mfirst ? 0 : -1;
#pragma unroll 4
    for (int f = fb; f < fe; ++f) {
      const V3<R> xf = s.cb(f, c);
      R e0, e1, e2 = 0, e21 = 0;
      if constexpr (sizeof(R) == 4) {
        const float u0 = bin_sat(dist_fast(xf, xm), tb), u1 = bin_sat(dist_fast(xf, y1), tb);
        float u2 = 1.f, u21 = 1.f;
        if (FUSED) {
          u2 = bin_sat(dist_fast(xf, y2), tb);
          u21 = bin_sat(dist_fast(xf, y21), tb);
        }
        // read nothing when every image is flat: the terms are then 0 - 0
        // instead of the flat value minus itself, the same exact zero
        const unsigned need = fminf(fminf(u0, u1), fminf(u2, u21)) < 1.f;
        nread += (need & live) << (FUSED ? 2 : 1);  // terms read
        if constexpr (TEX) {
          e0 = term_tex_if(rowe, u0, tb, need);
          e1 = term_tex_if(rowe, u1, tb, need);
          if (FUSED) {
            e2 = term_tex_if(rowe, u2, tb, need);
            e21 = term_tex_if(rowe, u21, tb, need);
          }
          rowe += step * tb.Bp;
        } else {
          e0 = term_ldg_if(row, u0, tb, need);
          e1 = term_ldg_if(row, u1, tb, need);
          if (FUSED) {
            e2 = term_ldg_if(row, u2, tb, need);
            e21 = term_ldg_if(row, u21, tb, need);
          }
          row += (long long)step * tb.Bp;
        }
      } else {
        e0 = pair_term(row, dist_fast(xf, xm), tb);
        e1 = pair_term(row, dist_fast(xf, y1), tb);
        if (FUSED) {
          e2 = pair_term(row, dist_fast(xf, y2), tb);
          e21 = pair_term(row, dist_fast(xf, y21), tb);
        }
        row += (long long)step * tb.Bp;
      }
      acc1 += e1 - e0;
      if (FUSED) {
        acc2 += e2 - e0;
        acc21 += e21 - e1;
      }
      step += dstep;
    }
  }
  if constexpr (sizeof(R) == 4)
    reduce3f(s, acc1, acc2, acc21);
  else
    reduce3(s, (double)acc1, (double)acc2, (double)acc21);
}

__device__ __forceinline__ float dist2(V3<float> a, V3<float> b) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  return fmaf(dz, dz, fmaf(dy, dy, dx * dx));
}
__device__ __forceinline__ V3<float> v3of(Pt4<float> p) { return v3<float>(p.x, p.y, p.z); }
__device__ __forceinline__ Pt4<float> pt4of(V3<float> v) {
  Pt4<float> p;
  p.x = v.x;
  p.y = v.y;
  p.z = v.z;
  p.w = 0.f;
  return p;
}

// Bounding spheres (box centre, largest distance) of the fixed side's
// kFC-atom chunks, one thread per (chunk, chain) among threads [t0, t0 + nt).
// They do not depend on the proposal, so warps other than the one drawing
// and rotating compute them meanwhile.
template <int C>
__device__ void far_spheres(Shm<float, C>& s, int f0, int f1, int t0, int nt) {
  const int nJ = (f1 - f0 + kFC - 1) / kFC;
  const Pt4<float>* __restrict__ cb4 = s.cb4;  // kept in registers for the loops
  Pt4<float>* __restrict__ fsph = s.fsph;
  const int ls = s.ls;
  for (int t = (int)threadIdx.x - t0; t < nJ * C; t += nt) {
    const int j = t / C, c = t - j * C;
    const int fb = f0 + kFC * j, fe = min(fb + kFC, f1);
    const Pt4<float>* x = cb4 + c * ls;
    V3<float> lo = v3of(x[fb]), hi = lo;
    for (int f = fb + 1; f < fe; ++f) {
      const Pt4<float> y = x[f];
      lo = v3<float>(fminf(lo.x, y.x), fminf(lo.y, y.y), fminf(lo.z, y.z));
      hi = v3<float>(fmaxf(hi.x, y.x), fmaxf(hi.y, y.y), fmaxf(hi.z, y.z));
    }
    const V3<float> o = (lo + hi) * 0.5f;
    float r2 = 0.f;
    for (int f = fb; f < fe; ++f) r2 = fmaxf(r2, dist2(v3of(x[f]), o));
    Pt4<float> q = pt4of(o);
    q.w = sqrtf(r2);
    fsph[j * C + c] = q;
  }
}

// The straddle block without its flat far field (FP32).  Beyond the last
// bin centre the Eq. 5 term is the constant -ln p of the last bin, so a pair
// whose distance is past it before and after the move adds exactly zero to
// Delta-E.  Per chain, the fixed side is cut into the kFC-atom chunks of the
// pair loop with bounding spheres, and each moving atom's images (the atom
// under A1, A2, A21) get one too; an item (moving atom, chunk) is run when
// the two spheres come within `cut` (the last centre plus a margin for
// rounding) for any chain of the CTA.  The kept items, listed in order, go
// through the same pair loop as the full block.
template <int C, bool FUSED, bool TEX>
__device__ void pair_block_far(Shm<float, C>& s, const Tab<float>& tb, long long tab_off, int L,
                               int m0, int m1, int f0, int f1, float cut, unsigned real,
                               unsigned long long& count, unsigned& nread) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  const int nM = m1 - m0, nJ = (f1 - f0 + kFC - 1) / kFC;
  const int nMs = s.nm;  // stride of s.bits per chain
  const Pt4<float>* __restrict__ fsph = s.fsph;
  ChunkBits* __restrict__ bits = s.bits;
  // (2) one thread per (moving atom, chain): the images' sphere and the
  // chunks within reach, as bits.  With one chain each thread takes the
  // contiguous range of moving atoms that it lists in (3), so it reads
  // back only its own bits and no barrier is needed between the two.
  const int per = (nM + blockDim.x - 1) / blockDim.x;
  const int b0 = min(nM, (int)threadIdx.x * per), b1 = min(nM, b0 + per);
  const int t_beg = C == 1 ? b0 : (int)threadIdx.x, t_end = C == 1 ? b1 : nM * C;
  const int t_step = C == 1 ? 1 : (int)blockDim.x;
  for (int t = t_beg; t < t_end; t += t_step) {
    const int mi = t / C, c = t - mi * C;
    ChunkBits b = 0;
    if ((real >> c) & 1u) {
      const V3<float> xm = s.cb(m0 + mi, c);
      Move<float> A;
      load_rot(s.maps + 36 * c, A);
      const V3<float> y1 = move_apply(A, xm);
      V3<float> o;
      float r2;
      if (FUSED) {
        load_move21(s.maps + 36 * c + 24, A.p, A);
        const V3<float> y21 = move_apply(A, xm);
        load_rot(s.maps + 36 * c + 12, A);
        const V3<float> y2 = move_apply(A, xm);
        o = (xm + y1 + y2 + y21) * 0.25f;
        r2 = fmaxf(fmaxf(dist2(xm, o), dist2(y1, o)), fmaxf(dist2(y2, o), dist2(y21, o)));
      } else {
        o = (xm + y1) * 0.5f;
        r2 = fmaxf(dist2(xm, o), dist2(y1, o));
      }
      const float reach = sqrtf(r2) + cut;
      for (int j = 0; j < nJ; ++j) {
        const Pt4<float> q = fsph[j * C + c];
        const float lim = reach + q.w;
        if (dist2(o, v3of(q)) < lim * lim) b |= ChunkBits(1) << j;
      }
    }
    bits[c * nMs + mi] = b;
  }
  if constexpr (C > 1) __syncthreads();
  // (3) the items kept for any chain, in item order (a block-wide scan of
  // their counts per moving atom)
  auto kept = [&](int mi) {
    ChunkBits w = 0;
#pragma unroll
    for (int c = 0; c < C; ++c) w |= bits[c * nMs + mi];
    return w;
  };
  int mine = 0;
  for (int mi = b0; mi < b1; ++mi) mine += __popcll(kept(mi));
  int incl = mine;
#pragma unroll
  for (int off = 1; off < 32; off <<= 1) {
    const int o = __shfl_up_sync(0xffffffffu, incl, off);
    if (lane >= off) incl += o;
  }
  int* wsum = reinterpret_cast<int*>(s.scan);  // warp totals (the scan area is free here)
  if (lane == 31) wsum[warp] = incl;
  __syncthreads();
  int base = 0, total = 0;
  for (int w = 0; w < W; ++w) {
    const int v = wsum[w];
    if (w < warp) base += v;
    total += v;
  }
  int q = base + incl - mine;
  for (int mi = b0; mi < b1; ++mi) {
    ChunkBits w = kept(mi);
    while (w) {
      const int j = __ffsll((long long)w) - 1;
      w &= w - 1;
      s.list[q++] = (unsigned short)(mi * nJ + j);
      count += (unsigned long long)min(kFC, f1 - f0 - kFC * j) * __popc(real) * (FUSED ? 4 : 2);
    }
  }
  __syncthreads();
  // (4) the kept items through the full block's pair loop
  pair_block<float, C, FUSED, TEX, true>(s, tb, tab_off, L, m0, m1, f0, f1, real, nread, s.list,
                                         total);
}

// The straddle block with its table rows staged in shared memory.  Each warp
// owns a ring of D slots; a slot holds the S = 32/C rows (one per slice) of
// one pair-iteration and completes on its own mbarrier.  Work items are
// (group of S moving atoms, chunk of fixed atoms): slice s takes moving
// atom m = group + s and all slices of a warp walk the same fixed atoms, so
// the warp's control flow is uniform.  A fetch cursor runs D iterations
// ahead of the compute cursor; lane 0 of each slice issues the bulk copy of
// its row.  Returns false (after flagging) if a wait gave up.
struct RowCursor {
  int it, f, fe, mb;   // item, fixed atom, end of chunk, first moving atom of the group
  const float2* row;   // this lane's row (f, mb + slice)
  int step, dstep;
  bool valid;
};

template <int C>
__device__ __forceinline__ void cursor_setup(RowCursor& k, int it, int items, int nch, int m0,
                                             int m1, int f0, int f1, int L, int sl,
                                             const float2* tab, int Bp) {
  constexpr int S = 32 / C;
  k.it = it;
  k.valid = it < items;
  if (!k.valid) return;
  const int g = it / nch, ch = it - g * nch;
  k.mb = m0 + g * S;
  k.f = f0 + ch * kFC;
  k.fe = min(k.f + kFC, f1);
  const int m = k.mb + sl;
  if (m < m1) {
    const bool mfirst = m < k.f;
    k.row = tab + (long long)(mfirst ? row_of(L, m, k.f) : row_of(L, k.f, m)) * Bp;
    k.step = mfirst ? 1 : L - k.f - 2;
    k.dstep = mfirst ? 0 : -1;
  }
}

template <int C, bool FUSED>
__device__ bool pair_block_staged(Shm<float, C>& s, const Tab<float>& tb, long long tab_off, int L,
                                  int m0, int m1, int f0, int f1, int D, unsigned& par,
                                  int* err, int wait_test) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, W = blockDim.x >> 5;
  constexpr int S = 32 / C;
  const int c = lane % C, sl = lane / C;
  const int Bp = tb.Bp;
  const int RB = Bp * (int)sizeof(float2);
  const float2* tab = tb.E + tab_off;
  Move<float> A1, A2, A21;
  load_rot(s.maps + 36 * c, A1);
  if (FUSED) {
    load_rot(s.maps + 36 * c + 12, A2);
    load_move21(s.maps + 36 * c + 24, A1.p, A21);
  }
  const int nF = f1 - f0;
  const int nch = (nF + kFC - 1) / kFC;
  const int nmg = (m1 - m0 + S - 1) / S;
  const int items = nmg * nch;
  const uint32_t ring = smem_addr(s.ring + (size_t)warp * D * S * RB);
  const uint32_t bar0 = smem_addr(s.bars + (size_t)warp * D);
  if (wait_test > 0) {
    // test hook: wait on slot 0 before any copy is issued; nothing can
    // complete its phase, so the wait gives up with no copy in flight
    const bool got = mbar_wait_tries(bar0, par & 1u, wait_test);
    if (!__all_sync(0xffffffffu, got)) {
      if (lane == 0) atomicOr(err, 2);
      reduce3f(s, 0.f, 0.f, 0.f);
      return false;
    }
  }

  RowCursor F;
  cursor_setup<C>(F, warp, items, nch, m0, m1, f0, f1, L, sl, tab, Bp);
  int qf = 0;
  // issue the copies of the fetch cursor's iteration into slot qf % D
  auto issue = [&]() {
    const int slot = qf % D;
    const uint32_t bar = bar0 + 8u * slot;
    const int nact = min(S, m1 - F.mb);
    if (lane == 0) mbar_arrive_expect_tx(bar, (unsigned)(nact * RB));
    __syncwarp();
    if (c == 0 && F.mb + sl < m1) {
      fence_proxy_async_smem();
      bulk_g2s(ring + (uint32_t)((slot * S + sl) * RB), F.row, (unsigned)RB, bar);
    }
    ++qf;
    if (F.f + 1 < F.fe) {
      ++F.f;
      F.row += (long long)F.step * Bp;
      F.step += F.dstep;
    } else {
      cursor_setup<C>(F, F.it + W, items, nch, m0, m1, f0, f1, L, sl, tab, Bp);
    }
  };
  for (int d = 0; d < D && F.valid; ++d) issue();

  float acc1 = 0.f, acc2 = 0.f, acc21 = 0.f;
  int q = 0;
  bool ok = true;
  for (int it = warp; it < items && ok; it += W) {
    const int g = it / nch, ch = it - g * nch;
    const int m = m0 + g * S + sl;
    const bool act = m < m1;
    V3<float> xm = v3<float>(0.f, 0.f, 0.f), y1 = xm, y2 = xm, y21 = xm;
    if (act) {
      xm = s.cb(m, c);
      y1 = move_apply(A1, xm);
      if (FUSED) {
        y2 = move_apply(A2, xm);
        y21 = move_apply(A21, xm);
      }
    }
    const int fb = f0 + ch * kFC, fe = min(fb + kFC, f1);
    for (int f = fb; f < fe; ++f) {
      const int slot = q % D;
      const bool got = mbar_wait_bounded(bar0 + 8u * slot, (par >> slot) & 1u);
      if (!__all_sync(0xffffffffu, got)) {
        ok = false;
        break;
      }
      par ^= 1u << slot;
      if (act) {
        const V3<float> xf = s.cb(f, c);
        const uint32_t srow = ring + (uint32_t)((slot * S + sl) * RB);
        const float e0 = pair_term_smem(srow, dist_(xf, xm), tb);
        const float e1 = pair_term_smem(srow, dist_(xf, y1), tb);
        acc1 += e1 - e0;
        if (FUSED) {
          const float e2 = pair_term_smem(srow, dist_(xf, y2), tb);
          const float e21 = pair_term_smem(srow, dist_(xf, y21), tb);
          acc2 += e2 - e0;
          acc21 += e21 - e1;
        }
      }
      __syncwarp();
      ++q;
      if (F.valid) issue();
    }
  }
  if (!ok) {
    // a copy did not arrive: flag it and wait (bounded) for the copies still
    // in flight before the slots are given up
    if (lane == 0) atomicOr(err, 2);
    for (; q < qf; ++q) {
      const int slot = q % D;
      mbar_wait_bounded(bar0 + 8u * slot, (par >> slot) & 1u);
      par ^= 1u << slot;
    }
  }
  reduce3f(s, acc1, acc2, acc21);
  return ok;
}

// Apply each chain's committed map to its moving residues [m0, m1).
template <class R, int C>
__device__ void commit_moves(Shm<R, C>& s, int m0, int m1, bool cb_only) {
  // cb_only: the upstream side moved; the rest of this sweep rotates about
  // bonds at or after the pivot and never reads these residues' torsion
  // axes (a new sweep starts from a rebuild), so only the C-betas move
  const int per = cb_only ? 1 : 4;
  const int total = (m1 - m0) * per * C;
  // the block size is a multiple of C: a thread's items all belong to
  // chain slot threadIdx.x % C, so it loads that slot's move once
  const int c = threadIdx.x % C;
  const int code = s.commit[c];
  if (!code) return;
  Move<R> A;
  if (code < 3)
    load_rot(s.maps + 36 * c + 12 * (code - 1), A);
  else
    load_move21(s.maps + 36 * c + 24, s.maps + 36 * c + 9, A);
  for (int idx = threadIdx.x; idx < total; idx += blockDim.x) {
    const int rest = idx / C;
    const int v = cb_only ? 3 : rest & 3, i = m0 + (cb_only ? rest : rest >> 2);
    if (v == 0) {
      s.set_bbv(i, 0, c, move_apply(A, s.bbv(i, 0, c)));
    } else if (v < 3) {
      s.set_bbv(i, v, c, move_lin(A, s.bbv(i, v, c)));
    } else {
      s.set_cb(i, c, move_apply(A, s.cb(i, c)));
    }
  }
}

// Temperature of chain slot c: T, times its ladder factor under parallel
// tempering.
template <class R>
__device__ __forceinline__ double chain_T(const SweepArgs<R>& a, const ProteinDev& P, int chain,
                                          double T) {
  return a.ladder ? T * a.ladder[(chain - P.chain0) % a.ladder_K] : T;
}

template <class R>
__device__ __forceinline__ void put_trace(const SweepArgs<R>& a, bool real, int chain, long long v,
                                          int k, int acc, R thn, R lnu, double dE) {
  if (real && chain < a.trace_chains && v < a.trace_cap) {
    TraceRec r;
    r.k = k;
    r.accept = acc;
    r.theta_new = (double)thn;
    r.lnu = (double)lnu;
    r.dE = dE;
    a.trace[(size_t)chain * a.trace_cap + v] = r;
  }
}

template <class R, int C>
__device__ void load_group(Shm<R, C>& s, const SweepArgs<R>& a, const GroupDev& G,
                           const ProteinDev& P) {
  const int n = P.n;
  for (int idx = threadIdx.x; idx < n * C; idx += blockDim.x) {
    const int c = idx / n, k = idx - c * n;
    R v = R(0);
    if (c < G.nchains) v = a.theta[P.tors0 + (long long)(G.chain0 - P.chain0 + c) * n + k];
    s.theta[k * C + c] = v;
  }
  if (threadIdx.x < C) s.acc[threadIdx.x] = 0;
}

// The chain slots' C-betas to the context's coordinate buffer (if kept).
template <class R, int C>
__device__ void store_coords(Shm<R, C>& s, const SweepArgs<R>& a, const GroupDev& G,
                             const ProteinDev& P) {
  if (!a.coords) return;
  const int L = P.L;
  for (int idx = threadIdx.x; idx < L * C; idx += blockDim.x) {
    const int c = idx / L, i = idx - c * L;
    if (c >= G.nchains) continue;
    const long long off = 3 * ((P.tors0 + (long long)(G.chain0 - P.chain0 + c) * P.n) / 2 + i);
    const V3<R> x = s.cb(i, c);
    a.coords[off] = x.x;
    a.coords[off + 1] = x.y;
    a.coords[off + 2] = x.z;
  }
}

// Write back torsions, counters, energies, accepted counts and best states.
template <class R, int C>
__device__ void store_group(Shm<R, C>& s, const SweepArgs<R>& a, const GroupDev& G,
                            const ProteinDev& P, long long t_end, bool update_best) {
  const int n = P.n;
  if (threadIdx.x < C) {
    const int c = threadIdx.x;
    int better = 0;
    if (c < G.nchains) {
      const int chain = G.chain0 + c;
      const double e = s.ecur[c];
      if (!(e == e)) atomicOr(a.err, 1);  // NaN energy
      a.E_cur[chain] = e;
      a.tcount[chain] = t_end;
      if (a.acc_out) a.acc_out[chain] = s.acc[c];
      if (a.trace_count && chain < a.trace_chains)
        a.trace_count[chain] = t_end < a.trace_cap ? t_end : a.trace_cap;
      if (update_best && e < a.best_E[chain]) {
        a.best_E[chain] = e;
        better = 1;
      }
    }
    s.flag[c] = better;
  }
  __syncthreads();
  for (int idx = threadIdx.x; idx < n * C; idx += blockDim.x) {
    const int c = idx / n, k = idx - c * n;
    if (c >= G.nchains) continue;
    const long long off = P.tors0 + (long long)(G.chain0 - P.chain0 + c) * n + k;
    const R v = s.theta[k * C + c];
    a.theta[off] = v;
    if (s.flag[c]) a.best_theta[off] = v;
  }
}

// Add the table terms read by a warp's lanes since the last flush to the
// context's counter (called by every thread of the CTA).
__device__ __forceinline__ void flush_reads(unsigned& nread, unsigned long long* dst) {
  unsigned v = nread;
  nread = 0;
#pragma unroll
  for (int off = 16; off > 0; off >>= 1) v += __shfl_xor_sync(0xffffffffu, v, off);
  if ((threadIdx.x & 31) == 0 && v && dst) atomicAdd(dst, (unsigned long long)v);
}

template <class R, int C, bool ST>
__device__ void run_group(Shm<R, C>& s, const SweepArgs<R>& a, const GroupDev& G,
                          const ProteinDev& P, unsigned& par, int* abort_flag) {
  const int L = P.L, n = P.n;
  load_group(s, a, G, P);
  const long long t0 = a.tcount[G.chain0];
  const long long steps = a.steps_are_sweeps ? a.steps * n : a.steps;
  // decisions need Delta-E only and the exit recomputes V from scratch, so
  // the entry and periodic resyncs rebuild the coordinates alone
  rebuild(s, a, P);
  long long since = 0;
  const unsigned real = G.nchains >= 32 ? ~0u : (1u << G.nchains) - 1u;  // slots holding chains
  unsigned long long count = 0;  // straddle terms whose distances this thread counted as formed
  unsigned nread = 0;            // FP32 terms whose entries this thread read
  long long d0 = 0, dend = 0;  // proposals [d0, dend) have their draws in s.draws
  int kn = (int)(t0 % n);      // torsion index of proposal t0 + j (kept without a 64-bit modulo)
  long long sw = 0;            // sweep of the call (scheduled calls start on a sweep boundary)
  double Tsw = a.T_of(0);
  // the temperature of this thread's chain slot in the form's precision
  // (threads below C take the decisions), formed once per sweep
  R Tc = (R)chain_T(a, P, G.chain0 + (int)(threadIdx.x % C), Tsw);
  R sig = a.sigma_of(0);
  for (long long j = 0; j < steps;) {
    const long long t = t0 + j;
    const int k = kn;
    if (k == 0 && j > 0 && a.nsched) {
      ++sw;
      Tsw = a.T_of(sw);
      Tc = (R)chain_T(a, P, G.chain0 + (int)(threadIdx.x % C), Tsw);
      sig = a.sigma_of(sw);
    }
    if (j + 2 > dend) {
      // the next proposals of this sweep (up to kDraw), made ahead by all
      // threads: their Philox draws depend on the counter only, and the
      // torsion each one changes is touched by no other proposal of the
      // sweep, so its value is final now.  The proposed value and the sine
      // and cosine of the rotation (signed for the side that moves) are
      // stored; the serial step keeps only the maps.
      __syncthreads();
      if (a.pair_count) flush_reads(nread, a.pair_count + 1);
      d0 = j;
      const int nb = min(kDraw, n - k);
      dend = j + nb;
      for (int idx = threadIdx.x; idx < nb * C; idx += blockDim.x) {
        const int q = idx / C, c = idx - q * C;
        const int kq = k + q;
        R z, lnu;
        normal_and_lnu(draw_words(a.seed, (uint32_t)(G.chain0 + c),
                                  (unsigned long long)(t0 + j + q), 0u),
                       &z, &lnu);
        const R th = s.theta[kq * C + c];
        const R thn = propose(th, z, sig, a.lattice_K);
        const R d = wrap_angle(thn - th);
        const int pq = (kq + 1) >> 1;
        R sn, cs;
        sincos_(pq <= L - pq ? -d : d, &sn, &cs);
        R* dr = s.draws + 4 * idx;
        dr[0] = thn;
        dr[1] = lnu;
        dr[2] = sn;
        dr[3] = cs;
      }
      __syncthreads();
    }
    // periodic rebuild, and one at each new sweep inside a call (commits of
    // upstream moves leave torsion axes behind, see commit_moves)
    if (since >= a.resync_every || (k == 0 && j > 0)) {
      rebuild(s, a, P);
      since = 0;
    }
    const bool fused = (k & 1) && (k + 1 < n) && (j + 1 < steps);
    const int p = (k + 1) >> 1;
    const bool up = p <= L - p;  // move the upstream side (it is the smaller)
    const int m0 = up ? 0 : p, m1 = up ? p : L;
    const int f0 = up ? p : 0, f1 = up ? L : p;
    const bool dead = (k == 0) || (k == n - 1);
    if constexpr (sizeof(R) == 4 && !ST) {
      // the far-field test's chunk spheres, by the warps that do not draw
      if (a.far_skip && !dead && threadIdx.x >= 32)
        far_spheres<C>(s, f0, f1, 32, (int)blockDim.x - 32);
    }
    if constexpr (C == 1) {
      // one chain: three lanes share the serial step.  Lane 0 makes move 1's
      // map A1, lane 1 move 2's map A2 about its own axis, lane 2 A1 again
      // and then the map of move 2 about the axis as move 1 left it,
      // composed after A1: the arithmetic of the one-lane form below in
      // two thirds of its latency (with more chains per CTA the split
      // measured slower)
      const int q = threadIdx.x;
      if (q == 0 || (q < 3 && fused)) {
        const int k1 = q == 1 ? k + 1 : k;
        const R* dr = s.draws + 4 * (j + (k1 - k) - d0);
        if (q < 2) {
          s.thn[q] = dr[0];
          s.lnu[q] = dr[1];
        }
        if (!dead) {
          // k1 odd: psi_i about CA_i -> C_i; k1 even: phi_i about N_i -> CA_i
          const int i = k1 >> 1;
          const Move<R> A =
              move_rotation_cs(s.bbv(i, 0, 0), s.bbv(i, (k1 & 1) ? 2 : 1, 0), dr[2], dr[3]);
          if (q < 2) {
            store_move(s.maps + 12 * q, A, A.p);
          } else {
            const R* dr2 = s.draws + 4 * (j + 1 - d0);
            const V3<R> P2 = s.bbv(p, 0, 0), u2 = s.bbv(p, 1, 0);  // phi_p: N_p -> CA_p
            // after move 1 the axis of move 2 has moved with the far side
            const V3<R> P2m = up ? P2 : move_apply(A, P2);
            const V3<R> u2m = up ? u2 : move_lin(A, u2);
            const Move<R> A21 = move_compose(move_rotation_cs(P2m, u2m, dr2[2], dr2[3]), A);
            store_move(s.maps + 24, A21, A21.q);
          }
        }
      }
    } else {
      if (threadIdx.x < C) {
        const int c = threadIdx.x;
        const R* dr = s.draws + 4 * ((j - d0) * C + c);
        s.thn[c] = dr[0];
        s.lnu[c] = dr[1];
        if (!dead) {
          // k odd: psi_i about CA_i -> C_i; k even: phi_i about N_i -> CA_i
          const int i = k >> 1;
          const Move<R> A1 =
              move_rotation_cs(s.bbv(i, 0, c), s.bbv(i, (k & 1) ? 2 : 1, c), dr[2], dr[3]);
          store_move(s.maps + 36 * c, A1, A1.p);
          if (fused) {
            const R* dr2 = s.draws + 4 * ((j + 1 - d0) * C + c);
            s.thn[C + c] = dr2[0];
            s.lnu[C + c] = dr2[1];
            const V3<R> P2 = s.bbv(p, 0, c), u2 = s.bbv(p, 1, c);  // phi_p: N_p -> CA_p
            const Move<R> A2 = move_rotation_cs(P2, u2, dr2[2], dr2[3]);
            store_move(s.maps + 36 * c + 12, A2, A2.p);
            // after move 1 the axis of move 2 has moved with the far side
            const V3<R> P2m = up ? P2 : move_apply(A1, P2);
            const V3<R> u2m = up ? u2 : move_lin(A1, u2);
            const Move<R> A2m = move_rotation_cs(P2m, u2m, dr2[2], dr2[3]);
            const Move<R> A21 = move_compose(A2m, A1);
            store_move(s.maps + 36 * c + 24, A21, A21.q);
          }
        }
      }
    }
    __syncthreads();
    if (dead) {
      // phi_0 and psi_{L-1} move no C-beta: Delta-E = 0, always accepted
      if (threadIdx.x < C) {
        const int c = threadIdx.x;
        const int chain = G.chain0 + c;
        const int acc = s.lnu[c] * Tc < -R(0);
        if (acc) s.theta[k * C + c] = s.thn[c];
        s.acc[c] += acc;
        put_trace(a, c < G.nchains, chain, t, k, acc, s.thn[c], s.lnu[c], 0.0);
      }
      __syncthreads();
      j += 1;
      since += 1;
      kn = k + 1 < n ? k + 1 : 0;
      continue;
    }
    if constexpr (ST) {
      const bool ok =
          fused ? pair_block_staged<C, true>(s, a.tab, P.tab_off, L, m0, m1, f0, f1,
                                             a.stage_depth, par, a.err, a.wait_test)
                : pair_block_staged<C, false>(s, a.tab, P.tab_off, L, m0, m1, f0, f1,
                                              a.stage_depth, par, a.err, a.wait_test);
      if (!ok) *(volatile int*)abort_flag = 1;
    } else if constexpr (sizeof(R) == 4) {
      if (a.far_skip) {
        if (a.tab.tex) {
          if (fused)
            pair_block_far<C, true, true>(s, a.tab, P.tab_off, L, m0, m1, f0, f1, a.far_cut, real,
                                          count, nread);
          else
            pair_block_far<C, false, true>(s, a.tab, P.tab_off, L, m0, m1, f0, f1, a.far_cut, real,
                                           count, nread);
        } else {
          if (fused)
            pair_block_far<C, true, false>(s, a.tab, P.tab_off, L, m0, m1, f0, f1, a.far_cut, real,
                                           count, nread);
          else
            pair_block_far<C, false, false>(s, a.tab, P.tab_off, L, m0, m1, f0, f1, a.far_cut, real,
                                            count, nread);
        }
      } else if (a.tab.tex) {
        if (fused)
          pair_block<R, C, true, true>(s, a.tab, P.tab_off, L, m0, m1, f0, f1, real, nread);
        else
          pair_block<R, C, false, true>(s, a.tab, P.tab_off, L, m0, m1, f0, f1, real, nread);
      } else {
        if (fused)
          pair_block<R, C, true, false>(s, a.tab, P.tab_off, L, m0, m1, f0, f1, real, nread);
        else
          pair_block<R, C, false, false>(s, a.tab, P.tab_off, L, m0, m1, f0, f1, real, nread);
      }
    } else {
      if (fused)
        pair_block<R, C, true, false>(s, a.tab, P.tab_off, L, m0, m1, f0, f1, real, nread);
      else
        pair_block<R, C, false, false>(s, a.tab, P.tab_off, L, m0, m1, f0, f1, real, nread);
    }
    if (threadIdx.x == 0 && !(sizeof(R) == 4 && !ST && a.far_skip))
      count += (unsigned long long)(m1 - m0) * (f1 - f0) * min(G.nchains, C) * (fused ? 4 : 2);
    __syncthreads();
    if (*(volatile int*)abort_flag) break;  // a staging wait gave up: stop (flagged)
    if (threadIdx.x < C) {
      const int c = threadIdx.x;
      const int chain = G.chain0 + c;
      const int W = blockDim.x >> 5;
      // the partial sums over the warps: FP32 in the FP32 form (each partial
      // is an FP32 sum already), FP64 in the FP64 form
      typename AccT<R>::T d1 = 0, d2 = 0, d21 = 0;
      for (int w = 0; w < W; ++w) {
        if constexpr (sizeof(R) == 4) {
          const float* pp = s.partf + (size_t)(w * C + c) * 3;
          d1 += pp[0];
          d2 += pp[1];
          d21 += pp[2];
        } else {
          const double* pp = s.part + (size_t)(w * C + c) * 3;
          d1 += pp[0];
          d2 += pp[1];
          d21 += pp[2];
        }
      }
      // Eq. 1 with T > 0: ln u < -dE / T  <=>  T ln u < -dE (no division),
      // in the form's precision (FP32: the product's rounding, 6e-8
      // relative, is far inside the 1e-5 tie margin of the decisions; the
      // FP64 pipe runs at 1/64 of the FP32 rate here)
      const int acc1 = s.lnu[c] * Tc < -d1;
      int code = acc1;
      if (acc1) s.theta[k * C + c] = s.thn[c];
      put_trace(a, c < G.nchains, chain, t, k, acc1, s.thn[c], s.lnu[c], (double)d1);
      int acc2 = 0;
      if (fused) {
        const typename AccT<R>::T e2 = acc1 ? d21 : d2;
        acc2 = s.lnu[C + c] * Tc < -e2;
        if (acc2) {
          code = acc1 ? 3 : 2;
          s.theta[(k + 1) * C + c] = s.thn[C + c];
        }
        put_trace(a, c < G.nchains, chain, t + 1, k + 1, acc2, s.thn[C + c], s.lnu[C + c],
                  (double)e2);
      }
      s.acc[c] += acc1 + acc2;
      s.commit[c] = code;
    }
    __syncthreads();
    commit_moves(s, m0, m1, up);
    __syncthreads();
    j += fused ? 2 : 1;
    kn = k + (fused ? 2 : 1);
    if (kn >= n) kn -= n;
    since += fused ? 2 : 1;
  }
  // exit: the energy from scratch (FP64 sum); the FP32 form takes the
  // current coordinates (their drift since the entry rebuild is ~1e-5 A),
  // the FP64 form rebuilds G(s) as well
  if constexpr (sizeof(R) == 4) {
    __syncthreads();
    full_energy(s, a.tab, P.tab_off, L);
  } else {
    resync(s, a, P);
  }
  store_coords(s, a, G, P);
  store_group(s, a, G, P, t0 + steps, true);
  if (a.pair_count) {
    // FP64 and staged sweeps read every term they form
    if (sizeof(R) == 8 || ST) nread = 0;
    flush_reads(nread, a.pair_count + 1);
    if (count) {
      atomicAdd(a.pair_count, count);
      if (sizeof(R) == 8 || ST) atomicAdd(a.pair_count + 1, count);
    }
  }
}

template <class R, int C, bool ST>
__global__ void __launch_bounds__(512) global_kernel(SweepArgs<R> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_group;
  __shared__ int s_abort;
  const int W = blockDim.x >> 5;
  const int D = ST ? a.stage_depth : 0;
  const Layout<R, C> lay(a.Lmax, a.nmax, W, D, ST ? a.tab.Bp * (int)sizeof(typename Vec2<R>::T) : 0);
  Shm<R, C> s(smem, lay);
  if (threadIdx.x == 0) s_abort = 0;
  if (ST && (threadIdx.x & 31) == 0) {
    const int w = threadIdx.x >> 5;
    for (int d = 0; d < D; ++d) mbar_init(smem_addr(s.bars + w * D + d), 1u);
    mbar_init_fence();
  }
  unsigned par = 0;  // per warp: phase parity to wait for, one bit per slot
  residue_basis(a.geom64, s.kb);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_group = s_abort ? a.ngroups : atomicAdd(a.queue, 1);
    __syncthreads();
    const int g = s_group;
    if (g >= a.ngroups) break;
    const GroupDev G = a.groups[g];
    const ProteinDev P = a.prot[G.protein];
    run_group<R, C, ST>(s, a, G, P, par, &s_abort);
  }
}

template <class R, int C>
__global__ void __launch_bounds__(512) energy_kernel(SweepArgs<R> a) {
  extern __shared__ __align__(128) unsigned char smem[];
  __shared__ int s_group;
  const Layout<R, C> lay(a.Lmax, a.nmax, blockDim.x >> 5);
  Shm<R, C> s(smem, lay);
  residue_basis(a.geom64, s.kb);
  for (;;) {
    __syncthreads();
    if (threadIdx.x == 0) s_group = atomicAdd(a.queue, 1);
    __syncthreads();
    const int g = s_group;
    if (g >= a.ngroups) break;
    const GroupDev G = a.groups[g];
    const ProteinDev P = a.prot[G.protein];
    load_group(s, a, G, P);
    resync(s, a, P);
    store_coords(s, a, G, P);
    if (threadIdx.x < C && threadIdx.x < G.nchains) {
      const double e = s.ecur[threadIdx.x];
      if (!(e == e)) atomicOr(a.err, 1);
      a.E_cur[G.chain0 + threadIdx.x] = e;
    }
  }
}

}  // namespace

template <class R, int C>
size_t global_smem_bytes(int Lmax, int nmax, int threads, int stage_depth, int row_bytes) {
  return Layout<R, C>(Lmax, nmax, threads / 32, stage_depth, row_bytes).total;
}

template <class R, int C, bool ST>
cudaError_t global_set_smem(size_t optin) {
  cudaError_t e = allow_dynamic_smem(global_kernel<R, C, ST>, optin);
  if (e != cudaSuccess) return e;
  return allow_dynamic_smem(energy_kernel<R, C>, optin);
}

template <class R, int C, bool ST>
cudaError_t global_occupancy(int threads, size_t smem, int* per_sm) {
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(per_sm, global_kernel<R, C, ST>, threads,
                                                       smem);
}

template <class R, int C, bool ST>
cudaError_t launch_global(const SweepArgs<R>& a, int threads, int grid, cudaStream_t st) {
  const int D = ST ? a.stage_depth : 0;
  const size_t sm = global_smem_bytes<R, C>(a.Lmax, a.nmax, threads, D,
                                            ST ? a.tab.Bp * (int)sizeof(typename Vec2<R>::T) : 0);
  global_kernel<R, C, ST><<<grid, threads, sm, st>>>(a);
  return cudaGetLastError();
}

template <class R, int C>
cudaError_t launch_energy(const SweepArgs<R>& a, int threads, int grid, cudaStream_t st) {
  const size_t sm = global_smem_bytes<R, C>(a.Lmax, a.nmax, threads, 0, 0);
  energy_kernel<R, C><<<grid, threads, sm, st>>>(a);
  return cudaGetLastError();
}

#define AMH_INST(R, C)                                                                          \
  template size_t global_smem_bytes<R, C>(int, int, int, int, int);                            \
  template cudaError_t global_set_smem<R, C, false>(size_t);                                   \
  template cudaError_t global_occupancy<R, C, false>(int, size_t, int*);                       \
  template cudaError_t launch_global<R, C, false>(const SweepArgs<R>&, int, int, cudaStream_t); \
  template cudaError_t launch_energy<R, C>(const SweepArgs<R>&, int, int, cudaStream_t);
#define AMH_INST_ST(C)                                                                          \
  template cudaError_t global_set_smem<float, C, true>(size_t);                                \
  template cudaError_t global_occupancy<float, C, true>(int, size_t, int*);                    \
  template cudaError_t launch_global<float, C, true>(const SweepArgs<float>&, int, int,        \
                                                     cudaStream_t);

AMH_INST(float, 1)
AMH_INST(float, 2)
AMH_INST(float, 4)
AMH_INST(float, 8)
AMH_INST(double, 1)
AMH_INST(double, 2)
AMH_INST(double, 4)
AMH_INST_ST(4)
AMH_INST_ST(8)

}  // namespace amh
