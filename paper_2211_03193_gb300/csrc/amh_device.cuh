// amh_device.cuh -- device-side building blocks of the AMH kernels (sm_103a).
//
// Philox4x32-10 (Salmon et al., SC'11), Box-Muller, NeRF placement with
// ideal geometry (Parsons et al. 2005; the paper only says x = G(s),
// Sec. 2.1), rigid rotation about a bond axis (Sec. 2.4, "Proposal
// Generation"), and the interpolated -ln p pair term of Eq. 5.
#pragma once

#include <cstdint>
#include <cuda_runtime.h>

namespace amh {

// ------------------------------------------------------------------ types
template <class R>
struct V3 {
  R x, y, z;
};

template <class R>
__device__ __forceinline__ V3<R> v3(R x, R y, R z) {
  V3<R> r;
  r.x = x;
  r.y = y;
  r.z = z;
  return r;
}
template <class R>
__device__ __forceinline__ V3<R> operator-(V3<R> a, V3<R> b) {
  return v3<R>(a.x - b.x, a.y - b.y, a.z - b.z);
}
template <class R>
__device__ __forceinline__ V3<R> operator+(V3<R> a, V3<R> b) {
  return v3<R>(a.x + b.x, a.y + b.y, a.z + b.z);
}
template <class R>
__device__ __forceinline__ V3<R> operator*(V3<R> a, R s) {
  return v3<R>(a.x * s, a.y * s, a.z * s);
}
template <class R>
__device__ __forceinline__ R dot(V3<R> a, V3<R> b) {
  return a.x * b.x + a.y * b.y + a.z * b.z;
}
template <class R>
__device__ __forceinline__ V3<R> cross(V3<R> a, V3<R> b) {
  return v3<R>(a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x);
}

// Correctly rounded 1/sqrt for the builders (NeRF frames, rotation axes):
// they are off the hot loop, and approximate normalisations there bend the
// chain systematically.
__device__ __forceinline__ float rsqrt_(float x) { return __frsqrt_rn(x); }
__device__ __forceinline__ double rsqrt_(double x) { return rsqrt(x); }
__device__ __forceinline__ void sincos_(float a, float* s, float* c) { sincosf(a, s, c); }
__device__ __forceinline__ void sincos_(double a, double* s, double* c) { sincos(a, s, c); }

template <class R>
__device__ __forceinline__ V3<R> unit(V3<R> a) {
  return a * rsqrt_(dot(a, a));
}

// 1/sqrt(x) by the approximate MUFU instruction with denormals flushed
// (x >= 1e-30 here, so no denormal path is needed).
__device__ __forceinline__ float rsqrt_ftz(float x) {
  float r;
  asm("rsqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(x));
  return r;
}

// Euclidean distance.  FP32: d2 * rsqrt(d2) (one MUFU op), with 1e-30
// folded into the first FMA so coincident points give 0, not NaN; FP64: sqrt.
__device__ __forceinline__ float dist_(V3<float> a, V3<float> b) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const float d2 = fmaf(dz, dz, fmaf(dy, dy, fmaf(dx, dx, 1e-30f)));
  return d2 * rsqrt_ftz(d2);
}
__device__ __forceinline__ double dist_(V3<double> a, V3<double> b) {
  V3<double> d = a - b;
  return sqrt(dot(d, d));
}

// Distance through one approximate square root (sqrt.approx, relative error
// of the order of 2^-23, sqrt(0) = 0): the pair loops of the sweeps.  FP64
// falls back to sqrt.
__device__ __forceinline__ float dist_fast(V3<float> a, V3<float> b) {
  const float dx = a.x - b.x, dy = a.y - b.y, dz = a.z - b.z;
  const float d2 = fmaf(dz, dz, fmaf(dy, dy, dx * dx));
  float r;
  asm("sqrt.approx.ftz.f32 %0, %1;" : "=f"(r) : "f"(d2));
  return r;
}
__device__ __forceinline__ double dist_fast(V3<double> a, V3<double> b) { return dist_(a, b); }

// ------------------------------------------------------------------ geometry
// Ideal geometry as (-bond cos(angle), bond sin(angle)) pairs, filled on
// the host in double precision (see amh.h for the values).
template <class R>
struct Geom {
  R bNCA, bCAC;                  // N-CA, CA-C bond lengths (first residue)
  R cosNCAC, sinNCAC;            // N-CA-C angle
  R pN_c, pN_s;                  // N(i+1):  bond C-N,  angle CA-C-N
  R pCA_c, pCA_s;                // CA(i+1): bond N-CA, angle C-N-CA
  R pC_c, pC_s;                  // C(i+1):  bond CA-C, angle N-CA-C
  R pCB_c, pCB_s;                // CB:      bond CA-CB, angle C-CA-CB
  R cbT_c, cbT_s;                // CB improper dihedral N-C-CA-CB (cos, sin)
};

// Normalisation for short builds (window-local coordinates): FP32 uses the
// approximate MUFU reciprocal square root; errors cannot accumulate over a
// window of a few residues.
template <class R>
__device__ __forceinline__ V3<R> unit_short(V3<R> a) {
  return a * rsqrt_(dot(a, a));
}
template <>
__device__ __forceinline__ V3<float> unit_short<float>(V3<float> a) {
  return a * rsqrt_ftz(dot(a, a));
}

// NeRF: atom D bonded to C with the given (-b cos a, b sin a) and dihedral
// A-B-C-D of cosine ct and sine st.  SHORT selects the short-build
// normalisation.
template <class R, bool SHORT = false>
__device__ __forceinline__ V3<R> place(V3<R> A, V3<R> B, V3<R> C, R pc, R ps, R ct, R st) {
  V3<R> bc = SHORT ? unit_short(C - B) : unit(C - B);
  V3<R> nrm = SHORT ? unit_short(cross(B - A, bc)) : unit(cross(B - A, bc));
  V3<R> m = cross(nrm, bc);
  R py = ps * ct, pz = ps * st;
  return v3<R>(C.x + bc.x * pc + m.x * py + nrm.x * pz, C.y + bc.y * pc + m.y * py + nrm.y * pz,
               C.z + bc.z * pc + m.z * py + nrm.z * pz);
}

// Canonical frame of a chain's (or window's) first residue.
template <class R>
__device__ __forceinline__ void first_residue(const Geom<R>& g, V3<R>& N, V3<R>& CA, V3<R>& C) {
  N = v3<R>(R(0), R(0), R(0));
  CA = v3<R>(g.bNCA, R(0), R(0));
  C = v3<R>(g.bNCA - g.bCAC * g.cosNCAC, g.bCAC * g.sinNCAC, R(0));
}

// Next residue from the previous one: psi_i, omega = 180 deg, phi_{i+1}.
template <class R, bool SHORT = false>
__device__ __forceinline__ void next_residue(const Geom<R>& g, V3<R>& N, V3<R>& CA, V3<R>& C,
                                             R psi, R phi) {
  R sp, cp, sf, cf;
  sincos_(psi, &sp, &cp);
  sincos_(phi, &sf, &cf);
  V3<R> N1 = place<R, SHORT>(N, CA, C, g.pN_c, g.pN_s, cp, sp);
  V3<R> CA1 = place<R, SHORT>(CA, C, N1, g.pCA_c, g.pCA_s, R(-1), R(0));
  V3<R> C1 = place<R, SHORT>(C, N1, CA1, g.pC_c, g.pC_s, cf, sf);
  N = N1;
  CA = CA1;
  C = C1;
}

template <class R, bool SHORT = false>
__device__ __forceinline__ V3<R> cbeta(const Geom<R>& g, V3<R> N, V3<R> CA, V3<R> C) {
  return place<R, SHORT>(N, C, CA, g.pCB_c, g.pCB_s, g.cbT_c, g.cbT_s);
}

// Affine map x -> M x + t (M row-major), stored as 12 values.
template <class R>
struct Aff {
  R m[9];
  R t[3];
};

template <class R>
__device__ __forceinline__ V3<R> apply(const Aff<R>& A, V3<R> x) {
  return v3<R>(fma(A.m[0], x.x, fma(A.m[1], x.y, fma(A.m[2], x.z, A.t[0]))),
               fma(A.m[3], x.x, fma(A.m[4], x.y, fma(A.m[5], x.z, A.t[1]))),
               fma(A.m[6], x.x, fma(A.m[7], x.y, fma(A.m[8], x.z, A.t[2]))));
}

// Right-handed rotation about the line through P along the unit vector u,
// by the angle whose sine and cosine are s and c (rotation_axis: by the
// angle itself).  Raising a dihedral by delta turns the far-side atoms by
// +delta about the bond from its second to its third atom.
template <class R>
__device__ __forceinline__ Aff<R> rotation_axis_cs(V3<R> P, V3<R> u, R s, R c) {
  R oc = R(1) - c;
  Aff<R> A;
  A.m[0] = c + u.x * u.x * oc;
  A.m[1] = u.x * u.y * oc - u.z * s;
  A.m[2] = u.x * u.z * oc + u.y * s;
  A.m[3] = u.y * u.x * oc + u.z * s;
  A.m[4] = c + u.y * u.y * oc;
  A.m[5] = u.y * u.z * oc - u.x * s;
  A.m[6] = u.z * u.x * oc - u.y * s;
  A.m[7] = u.z * u.y * oc + u.x * s;
  A.m[8] = c + u.z * u.z * oc;
  // t = P - M P
  A.t[0] = P.x - (A.m[0] * P.x + A.m[1] * P.y + A.m[2] * P.z);
  A.t[1] = P.y - (A.m[3] * P.x + A.m[4] * P.y + A.m[5] * P.z);
  A.t[2] = P.z - (A.m[6] * P.x + A.m[7] * P.y + A.m[8] * P.z);
  return A;
}
template <class R>
__device__ __forceinline__ Aff<R> rotation_axis(V3<R> P, V3<R> u, R ang) {
  R s, c;
  sincos_(ang, &s, &c);
  return rotation_axis_cs(P, u, s, c);
}

// The same about the axis through P towards Q.
template <class R>
__device__ __forceinline__ Aff<R> rotation(V3<R> P, V3<R> Q, R ang) {
  return rotation_axis(P, unit(Q - P), ang);
}

// The linear part of A applied to a direction.
template <class R>
__device__ __forceinline__ V3<R> lin(const Aff<R>& A, V3<R> v) {
  return v3<R>(fma(A.m[0], v.x, fma(A.m[1], v.y, A.m[2] * v.z)),
               fma(A.m[3], v.x, fma(A.m[4], v.y, A.m[5] * v.z)),
               fma(A.m[6], v.x, fma(A.m[7], v.y, A.m[8] * v.z)));
}

// B o A (apply A first).
template <class R>
__device__ __forceinline__ Aff<R> compose(const Aff<R>& B, const Aff<R>& A) {
  Aff<R> r;
#pragma unroll
  for (int i = 0; i < 3; ++i) {
#pragma unroll
    for (int j = 0; j < 3; ++j)
      r.m[3 * i + j] = B.m[3 * i] * A.m[j] + B.m[3 * i + 1] * A.m[3 + j] + B.m[3 * i + 2] * A.m[6 + j];
    r.t[i] = B.m[3 * i] * A.t[0] + B.m[3 * i + 1] * A.t[1] + B.m[3 * i + 2] * A.t[2] + B.t[i];
  }
  return r;
}

// Four values at a 4-value boundary (one 16-byte shared load in FP32): a
// padded point, or a third of an affine map.
template <class R>
struct alignas(4 * sizeof(R)) Pt4 {
  R x, y, z, w;
};

// An affine map stored as three Pt4: m[0..3], m[4..7], (m[8], t).
template <class R>
__device__ __forceinline__ Aff<R> aff_load4(const Pt4<R>* q) {
  const Pt4<R> a = q[0], b = q[1], d = q[2];
  Aff<R> A;
  A.m[0] = a.x; A.m[1] = a.y; A.m[2] = a.z; A.m[3] = a.w;
  A.m[4] = b.x; A.m[5] = b.y; A.m[6] = b.z; A.m[7] = b.w;
  A.m[8] = d.x; A.t[0] = d.y; A.t[1] = d.z; A.t[2] = d.w;
  return A;
}

template <class R>
__device__ __forceinline__ void aff_store4(Pt4<R>* q, const Aff<R>& A) {
  Pt4<R> a, b, d;
  a.x = A.m[0]; a.y = A.m[1]; a.z = A.m[2]; a.w = A.m[3];
  b.x = A.m[4]; b.y = A.m[5]; b.z = A.m[6]; b.w = A.m[7];
  d.x = A.m[8]; d.y = A.t[0]; d.z = A.t[1]; d.w = A.t[2];
  q[0] = a;
  q[1] = b;
  q[2] = d;
}

template <class R>
__device__ __forceinline__ Aff<R> identity_map() {
  Aff<R> A;
#pragma unroll
  for (int i = 0; i < 9; ++i) A.m[i] = (i % 4 == 0) ? R(1) : R(0);
  A.t[0] = A.t[1] = A.t[2] = R(0);
  return A;
}

// ------------------------------------------------------------------ moves
// A proposal's rigid move, y = q + M (x - p): M a rotation, p a point and
// q its image.  Kept this way the FP32 rounding of p and q is that of one
// stored coordinate near the moving atoms.  The affine form x -> M x + t has
// t = p - M p rounded at the size of the coordinates (~1e-5 A at 50-80 A
// from the origin), one shift shared by the whole moving side, and Delta-E
// feels it with the net force on that side (~2e4 per A: up to ~0.2 for
// one move at L=150).
template <class R>
struct Move {
  R m[9];
  R p[3];
  R q[3];
};

// Rotation about the line through P along the unit vector u (right-handed;
// see rotation_axis_cs), by the angle of sine s and cosine c, or by `ang`.
template <class R>
__device__ __forceinline__ Move<R> move_rotation_cs(V3<R> P, V3<R> u, R s, R c) {
  const Aff<R> A = rotation_axis_cs(P, u, s, c);
  Move<R> M;
#pragma unroll
  for (int i = 0; i < 9; ++i) M.m[i] = A.m[i];
  M.p[0] = M.q[0] = P.x;
  M.p[1] = M.q[1] = P.y;
  M.p[2] = M.q[2] = P.z;
  return M;
}
template <class R>
__device__ __forceinline__ Move<R> move_rotation(V3<R> P, V3<R> u, R ang) {
  R s, c;
  sincos_(ang, &s, &c);
  return move_rotation_cs(P, u, s, c);
}

template <class R>
__device__ __forceinline__ V3<R> move_lin(const Move<R>& A, V3<R> v) {
  return v3<R>(fma(A.m[0], v.x, fma(A.m[1], v.y, A.m[2] * v.z)),
               fma(A.m[3], v.x, fma(A.m[4], v.y, A.m[5] * v.z)),
               fma(A.m[6], v.x, fma(A.m[7], v.y, A.m[8] * v.z)));
}

template <class R>
__device__ __forceinline__ V3<R> move_apply(const Move<R>& A, V3<R> x) {
  const R dx = x.x - A.p[0], dy = x.y - A.p[1], dz = x.z - A.p[2];
  return v3<R>(fma(A.m[0], dx, fma(A.m[1], dy, fma(A.m[2], dz, A.q[0]))),
               fma(A.m[3], dx, fma(A.m[4], dy, fma(A.m[5], dz, A.q[1]))),
               fma(A.m[6], dx, fma(A.m[7], dy, fma(A.m[8], dz, A.q[2]))));
}

// B o A (apply A first): taken about A's point, which lands on B(A(p)).
template <class R>
__device__ __forceinline__ Move<R> move_compose(const Move<R>& B, const Move<R>& A) {
  Move<R> r;
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      r.m[3 * i + j] = B.m[3 * i] * A.m[j] + B.m[3 * i + 1] * A.m[3 + j] + B.m[3 * i + 2] * A.m[6 + j];
  const V3<R> q = move_apply(B, v3<R>(A.q[0], A.q[1], A.q[2]));
  r.p[0] = A.p[0]; r.p[1] = A.p[1]; r.p[2] = A.p[2];
  r.q[0] = q.x; r.q[1] = q.y; r.q[2] = q.z;
  return r;
}

// A maps region holds A1, A2 and A21 as 12 values each at a 4-value
// boundary (three vector loads): the rotations' M and p (their q is
// p), and for A21 its M and q; its p is A1's (move 1's axis point).
template <class R>
__device__ __forceinline__ void load_rot(const R* src, Move<R>& A) {
  const Pt4<R>* v = reinterpret_cast<const Pt4<R>*>(src);
  const Pt4<R> a = v[0], b = v[1], d = v[2];
  A.m[0] = a.x; A.m[1] = a.y; A.m[2] = a.z; A.m[3] = a.w;
  A.m[4] = b.x; A.m[5] = b.y; A.m[6] = b.z; A.m[7] = b.w;
  A.m[8] = d.x; A.p[0] = A.q[0] = d.y; A.p[1] = A.q[1] = d.z; A.p[2] = A.q[2] = d.w;
}

// A21 from its 12 values and A1's point p1.
template <class R>
__device__ __forceinline__ void load_move21(const R* src, const R* p1, Move<R>& A) {
  const Pt4<R>* v = reinterpret_cast<const Pt4<R>*>(src);
  const Pt4<R> a = v[0], b = v[1], d = v[2];
  A.m[0] = a.x; A.m[1] = a.y; A.m[2] = a.z; A.m[3] = a.w;
  A.m[4] = b.x; A.m[5] = b.y; A.m[6] = b.z; A.m[7] = b.w;
  A.m[8] = d.x; A.q[0] = d.y; A.q[1] = d.z; A.q[2] = d.w;
  A.p[0] = p1[0]; A.p[1] = p1[1]; A.p[2] = p1[2];
}

// The 12 values of a rotation (pt = p) or of A21 (pt = q).
template <class R>
__device__ __forceinline__ void store_move(R* dst, const Move<R>& A, const R* pt) {
#pragma unroll
  for (int i = 0; i < 9; ++i) dst[i] = A.m[i];
#pragma unroll
  for (int i = 0; i < 3; ++i) dst[9 + i] = pt[i];
}

// ------------------------------------------------------------------ parallel G(s)
// Every residue is the same rigid body (ideal geometry), so G(s) is a chain
// of rigid transforms: with residue 0 in the canonical frame of
// first_residue(), residue i sits at P_i = T_1 o ... o T_i applied to the
// canonical atoms, where T_i (depending on psi_{i-1} and phi_i only) maps the
// canonical residue onto residue i as built by NeRF from a canonical residue
// i-1.  The T_i are computed independently and P_i is a prefix composition,
// evaluated here as a parallel scan in FP64.

// Orthonormal frame of a residue (columns e1 = CA->C, e2 = CA->N made
// orthogonal to e1, e3 = e1 x e2) as the rotation part of an affine map.
template <class R>
__device__ __forceinline__ void residue_frame(V3<R> N, V3<R> CA, V3<R> C, R Q[9]) {
  const V3<R> e1 = unit(C - CA);
  V3<R> v = N - CA;
  v = v - e1 * dot(v, e1);
  const V3<R> e2 = unit(v);
  const V3<R> e3 = cross(e1, e2);
  Q[0] = e1.x; Q[1] = e2.x; Q[2] = e3.x;
  Q[3] = e1.y; Q[4] = e2.y; Q[5] = e3.y;
  Q[6] = e1.z; Q[7] = e2.z; Q[8] = e3.z;
}

template <class R>
struct CanonicalResidue {
  V3<R> N, CA, C, CB;
  R Q0[9];  // frame of the canonical residue
};

template <class R>
__device__ __forceinline__ CanonicalResidue<R> canonical_residue(const Geom<R>& g) {
  CanonicalResidue<R> r;
  first_residue(g, r.N, r.CA, r.C);
  r.CB = cbeta(g, r.N, r.CA, r.C);
  residue_frame(r.N, r.CA, r.C, r.Q0);
  return r;
}

// T_i: canonical residue -> residue i in the frame of canonical residue i-1.
template <class R>
__device__ __forceinline__ Aff<R> residue_step(const Geom<R>& g, const CanonicalResidue<R>& r,
                                               R psi, R phi) {
  V3<R> N = r.N, CA = r.CA, C = r.C;
  next_residue(g, N, CA, C, psi, phi);
  R Q1[9];
  residue_frame(N, CA, C, Q1);
  Aff<R> T;
  // M = Q1 Q0^T, t = CA1 - M CA0
#pragma unroll
  for (int i = 0; i < 3; ++i)
#pragma unroll
    for (int j = 0; j < 3; ++j)
      T.m[3 * i + j] = Q1[3 * i] * r.Q0[3 * j] + Q1[3 * i + 1] * r.Q0[3 * j + 1] +
                       Q1[3 * i + 2] * r.Q0[3 * j + 2];
  T.t[0] = CA.x - (T.m[0] * r.CA.x + T.m[1] * r.CA.y + T.m[2] * r.CA.z);
  T.t[1] = CA.y - (T.m[3] * r.CA.x + T.m[4] * r.CA.y + T.m[5] * r.CA.z);
  T.t[2] = CA.z - (T.m[6] * r.CA.x + T.m[7] * r.CA.y + T.m[8] * r.CA.z);
  return T;
}

// T(psi, phi) = R_psi(psi) o T(0, 0) o R_phi(phi): changing psi_{i-1} turns
// residue i rigidly about a bond fixed in residue i-1's frame, changing
// phi_i turns residue i's frame about its own N-CA bond.  Each rotation is
// affine in (1, cos, sin), so T is bilinear in (1, cos psi, sin psi) x
// (1, cos phi, sin phi): T = sum_ab f_a(psi) g_b(phi) K_ab.  The nine K_ab
// follow from T on the grid {0, pi/2, pi}^2 (K_1 = (T(0) + T(pi))/2,
// K_cos = (T(0) - T(pi))/2, K_sin = T(pi/2) - K_1 per angle).
// residue_basis fills kb[0..108) with the K_ab (kb[108..216) is scratch);
// every thread of the CTA must call it.
__device__ inline void residue_basis(const Geom<double>& g, double* kb) {
  const double ang[3] = {0.0, 1.5707963267948966, 3.141592653589793};
  double* S = kb + 108;  // [9][12]: T at (psi_i, phi_j)
  if (threadIdx.x < 9) {
    const CanonicalResidue<double> cr = canonical_residue(g);
    const Aff<double> T = residue_step(g, cr, ang[threadIdx.x / 3], ang[threadIdx.x % 3]);
#pragma unroll
    for (int q = 0; q < 9; ++q) S[threadIdx.x * 12 + q] = T.m[q];
#pragma unroll
    for (int q = 0; q < 3; ++q) S[threadIdx.x * 12 + 9 + q] = T.t[q];
  }
  __syncthreads();
  if (threadIdx.x < 12) {
    const int q = threadIdx.x;
    double Y[3][3];  // [psi coefficient][phi sample]
    for (int j = 0; j < 3; ++j) {
      const double t0 = S[(0 * 3 + j) * 12 + q], t1 = S[(1 * 3 + j) * 12 + q],
                   t2 = S[(2 * 3 + j) * 12 + q];
      Y[0][j] = 0.5 * (t0 + t2);
      Y[1][j] = 0.5 * (t0 - t2);
      Y[2][j] = t1 - Y[0][j];
    }
    for (int a = 0; a < 3; ++a) {
      const double k0 = 0.5 * (Y[a][0] + Y[a][2]);
      kb[(a * 3 + 0) * 12 + q] = k0;
      kb[(a * 3 + 1) * 12 + q] = 0.5 * (Y[a][0] - Y[a][2]);
      kb[(a * 3 + 2) * 12 + q] = Y[a][1] - k0;
    }
  }
  __syncthreads();
}

// T_i from the basis of residue_basis: two sincos and 108 FMA.
__device__ __forceinline__ Aff<double> residue_step_basis(const double* kb, double psi,
                                                          double phi) {
  double sp, cp, sf, cf;
  sincos(psi, &sp, &cp);
  sincos(phi, &sf, &cf);
  const double f[3] = {1.0, cp, sp}, gg[3] = {1.0, cf, sf};
  double v[12];
#pragma unroll
  for (int q = 0; q < 12; ++q) v[q] = 0.0;
#pragma unroll
  for (int a = 0; a < 3; ++a)
#pragma unroll
    for (int b = 0; b < 3; ++b) {
      const double w = f[a] * gg[b];
      const double* K = kb + (a * 3 + b) * 12;
#pragma unroll
      for (int q = 0; q < 12; ++q) v[q] = fma(w, K[q], v[q]);
    }
  Aff<double> T;
#pragma unroll
  for (int q = 0; q < 9; ++q) T.m[q] = v[q];
#pragma unroll
  for (int q = 0; q < 3; ++q) T.t[q] = v[9 + q];
  return T;
}

__device__ __forceinline__ Aff<double> shfl_up_aff(const Aff<double>& A, int off, int width) {
  Aff<double> B;
#pragma unroll
  for (int i = 0; i < 9; ++i) B.m[i] = __shfl_up_sync(0xffffffffu, A.m[i], off, width);
#pragma unroll
  for (int i = 0; i < 3; ++i) B.t[i] = __shfl_up_sync(0xffffffffu, A.t[i], off, width);
  return B;
}

// Build G(s) of `nch` chains with the first nthreads threads of the CTA
// (0: all), kb the basis of residue_basis: chain c uses the tpc = nthreads / nslots consecutive threads
// starting at c * tpc (tpc a power of two).  theta(c, k) reads torsion k of
// chain c; emit(c, i, N, CA, C, CB) stores residue i.  scratch: nslots *
// max(tpc/32, 1) * 12 doubles of shared memory.  cache (optional, nslots * L
// * 12 doubles of shared memory) keeps each T_i so the second pass does not
// recompute it.  Must be called by every one of those threads; with tpc > 32
// it synchronises the whole CTA, so then nthreads must be the CTA.
template <class TH, class EMIT>
__device__ void build_chains_scan(const Geom<double>& g, const double* kb, int L, int nslots,
                                  TH theta, EMIT emit, double* scratch, double* cache = nullptr,
                                  int nthreads = 0) {
  const int tpc = (nthreads ? nthreads : (int)blockDim.x) / nslots;
  const int c = threadIdx.x / tpc, r = threadIdx.x % tpc;
  const int width = tpc < 32 ? tpc : 32;
  const int lane = r % width;
  const int wpc = tpc / width;  // warps per chain
  const int wi = r / width;     // this thread's warp within its chain
  const CanonicalResidue<double> cr = canonical_residue(g);
  const int nb = (L + tpc - 1) / tpc;
  const int r0 = min(L, r * nb), r1 = min(L, r0 + nb);
  Aff<double> agg = identity_map<double>();
  for (int i = max(r0, 1); i < r1; ++i) {
    const Aff<double> T = residue_step_basis(kb, theta(c, 2 * i - 1), theta(c, 2 * i));
    if (cache) {
      double* q = cache + ((size_t)c * L + i) * 12;
#pragma unroll
      for (int k = 0; k < 9; ++k) q[k] = T.m[k];
#pragma unroll
      for (int k = 0; k < 3; ++k) q[9 + k] = T.t[k];
    }
    agg = compose(agg, T);
  }
  // inclusive scan over the lanes of this chain's warp
  for (int off = 1; off < width; off <<= 1) {
    const Aff<double> o = shfl_up_aff(agg, off, width);
    if (lane >= off) agg = compose(o, agg);
  }
  Aff<double> excl = shfl_up_aff(agg, 1, width);
  if (lane == 0) excl = identity_map<double>();
  if (wpc > 1) {
    double* tot = scratch + (size_t)(c * wpc + wi) * 12;
    if (lane == width - 1) {
#pragma unroll
      for (int q = 0; q < 9; ++q) tot[q] = agg.m[q];
#pragma unroll
      for (int q = 0; q < 3; ++q) tot[9 + q] = agg.t[q];
    }
    __syncthreads();
    Aff<double> pre = identity_map<double>();
    for (int w = 0; w < wi; ++w) {
      const double* tw = scratch + (size_t)(c * wpc + w) * 12;
      Aff<double> A;
#pragma unroll
      for (int q = 0; q < 9; ++q) A.m[q] = tw[q];
#pragma unroll
      for (int q = 0; q < 3; ++q) A.t[q] = tw[9 + q];
      pre = compose(pre, A);
    }
    excl = compose(pre, excl);
    __syncthreads();
  }
  Aff<double> P = excl;
  for (int i = r0; i < r1; ++i) {
    if (i >= 1) {
      Aff<double> T;
      if (cache) {
        const double* q = cache + ((size_t)c * L + i) * 12;
#pragma unroll
        for (int k = 0; k < 9; ++k) T.m[k] = q[k];
#pragma unroll
        for (int k = 0; k < 3; ++k) T.t[k] = q[9 + k];
      } else {
        T = residue_step_basis(kb, theta(c, 2 * i - 1), theta(c, 2 * i));
      }
      P = compose(P, T);
    }
    emit(c, i, apply(P, cr.N), apply(P, cr.CA), apply(P, cr.C), apply(P, cr.CB));
  }
}

// The same build for one chain by nt threads (a multiple of 32; this one is
// t), whose warps meet at sync(): scratch holds nt/32 * 12 doubles.
template <class TH, class EMIT, class SYNC>
__device__ void build_chain_group(const Geom<double>& g, const double* kb, int L, int t, int nt,
                                  TH theta, EMIT emit, double* scratch, SYNC sync) {
  const int lane = t & 31, wi = t >> 5, wpc = nt >> 5;
  const CanonicalResidue<double> cr = canonical_residue(g);
  const int nb = (L + nt - 1) / nt;
  const int r0 = min(L, t * nb), r1 = min(L, r0 + nb);
  Aff<double> agg = identity_map<double>();
  for (int i = max(r0, 1); i < r1; ++i)
    agg = compose(agg, residue_step_basis(kb, theta(2 * i - 1), theta(2 * i)));
  for (int off = 1; off < 32; off <<= 1) {
    const Aff<double> o = shfl_up_aff(agg, off, 32);
    if (lane >= off) agg = compose(o, agg);
  }
  Aff<double> excl = shfl_up_aff(agg, 1, 32);
  if (lane == 0) excl = identity_map<double>();
  if (wpc > 1) {
    double* tot = scratch + (size_t)wi * 12;
    if (lane == 31) {
#pragma unroll
      for (int q = 0; q < 9; ++q) tot[q] = agg.m[q];
#pragma unroll
      for (int q = 0; q < 3; ++q) tot[9 + q] = agg.t[q];
    }
    sync();
    Aff<double> pre = identity_map<double>();
    for (int w = 0; w < wi; ++w) {
      const double* tw = scratch + (size_t)w * 12;
      Aff<double> A;
#pragma unroll
      for (int q = 0; q < 9; ++q) A.m[q] = tw[q];
#pragma unroll
      for (int q = 0; q < 3; ++q) A.t[q] = tw[9 + q];
      pre = compose(pre, A);
    }
    excl = compose(pre, excl);
    sync();
  }
  Aff<double> P = excl;
  for (int i = r0; i < r1; ++i) {
    if (i >= 1) P = compose(P, residue_step_basis(kb, theta(2 * i - 1), theta(2 * i)));
    emit(i, apply(P, cr.N), apply(P, cr.CA), apply(P, cr.C), apply(P, cr.CB));
  }
}

// ------------------------------------------------------------------ table
// Pair term of Eq. 5: -ln p interpolated linearly between evenly spaced bin
// centres c_j = c0 + j w, flat outside [c_0, c_{B-1}].  Each row holds one
// 8-byte entry per bin, so one load and one FMA give the term:
//  FP64: (E_j, E_{j+1} - E_j), term = E_j + (u - j) (E_{j+1} - E_j) with u the
//        bin coordinate (d - c0)/w clamped to [0, B-1];
//  FP32: (E_j - j D_j, (B-1) D_j), D_j = E_{j+1} - E_j, term = fmaf(us, .y,
//        .x) with us = u / (B-1) in [0, 1]: the same line, with j folded into
//        the entry so the term needs no fractional part.
// The last bin and the padding hold (E_{B-1}, 0).
template <class R>
struct Vec2;
template <>
struct Vec2<float> {
  using T = float2;
};
template <>
struct Vec2<double> {
  using T = double2;
};

template <class R>
struct Tab {
  const typename Vec2<R>::T* __restrict__ E;  // [rows][Bp] (value, slope per bin)
  R inv_w;                                    // 1 / w
  R off;                                      // -c0 / w
  R umax;                                     // B - 1
  R k1, k2;                                   // inv_w / umax, off / umax
  int Bp;
  cudaTextureObject_t tex;                    // FP32: the same entries as a 1-D texture (or 0)
};

// floor(u) for 0 <= u < 2^22 as (integer, float): adding 2^23 rounded down
// leaves floor(u) in the low mantissa bits (FP32 pipe only).
__device__ __forceinline__ int floor_small(float u, float* jf) {
  const float f = __fadd_rd(u, 8388608.0f);
  *jf = f - 8388608.0f;
  return __float_as_int(f) - 0x4B000000;
}
__device__ __forceinline__ int floor_small(double u, double* jf) {
  const int j = (int)u;
  *jf = (double)j;
  return j;
}

__device__ __forceinline__ double pair_term(const double2* __restrict__ row, double d,
                                            const Tab<double>& tb) {
  double u = fma(d, tb.inv_w, tb.off);
  u = fmin(fmax(u, 0.0), tb.umax);
  double jf;
  const int j = floor_small(u, &jf);
  const double2 v = __ldg(row + j);
  return fma(u - jf, v.y, v.x);
}

// FP32: the bin coordinate u = (d - c0)/w clamped to [0, B-1] is
// umax * sat(d k1 + k2) (one FFMA.SAT); floor(u) + 2^23 comes from one FMA
// rounded down, whose bit pattern also indexes the entry: bin j sits at
// byte 8 j of the row, i.e. at row - 8 * 0x4B000000 + 8 * bits.
__device__ __forceinline__ float pair_term(const float2* __restrict__ row, float d,
                                           const Tab<float>& tb) {
  const float us = __saturatef(fmaf(d, tb.k1, tb.k2));
  const float f = __fmaf_rd(us, tb.umax, 8388608.0f);
  const char* base = reinterpret_cast<const char*>(row) - 8ull * 0x4B000000u;
  float2 v;
  // one wide multiply-add forms the entry address from the float's bits
  asm("{\n\t.reg .u64 ad;\n\tmad.wide.u32 ad, %2, 8, %3;\n\t"
      "ld.global.nc.v2.f32 {%0, %1}, [ad];\n\t}"
      : "=f"(v.x), "=f"(v.y)
      : "r"((unsigned)__float_as_int(f)), "l"(base));
  return fmaf(us, v.y, v.x);
}

// Value and slope d e / d d (zero on the flat ends).
__device__ __forceinline__ double pair_term_slope(const double2* __restrict__ row, double d,
                                                  const Tab<double>& tb, double* slope) {
  const double u0 = fma(d, tb.inv_w, tb.off);
  const double u = fmin(fmax(u0, 0.0), tb.umax);
  double jf;
  const int j = floor_small(u, &jf);
  const double2 v = __ldg(row + j);
  *slope = (u0 >= 0.0 && u0 < tb.umax) ? v.y * tb.inv_w : 0.0;
  return fma(u - jf, v.y, v.x);
}
__device__ __forceinline__ float pair_term_slope(const float2* __restrict__ row, float d,
                                                 const Tab<float>& tb, float* slope) {
  const float s0 = fmaf(d, tb.k1, tb.k2);
  const float us = __saturatef(s0);
  const float f = __fmaf_rd(us, tb.umax, 8388608.0f);
  const float2 v = __ldg(row + (__float_as_int(f) - 0x4B000000));
  *slope = (s0 >= 0.f && s0 < 1.f) ? v.y * tb.k1 : 0.f;
  return fmaf(us, v.y, v.x);
}

// The same term fetched through the texture path from a 32-bit entry index
// (row_e: index of the row's first entry): the texture unit forms the
// address, so a term costs one integer add instead of 64-bit arithmetic.
__device__ __forceinline__ float pair_term_tex(int row_e, float d, const Tab<float>& tb) {
  const float us = __saturatef(fmaf(d, tb.k1, tb.k2));
  const float f = __fmaf_rd(us, tb.umax, 8388608.0f);
  const float2 v = tex1Dfetch<float2>(tb.tex, row_e - 0x4B000000 + __float_as_int(f));
  return fmaf(us, v.y, v.x);
}

// The FP32 term split in two, so that a pair can be tested before its entry
// is read.  bin_sat: the saturated bin coordinate us of a distance; us == 1
// exactly when d is at or past the last bin centre, where every distance of
// the row reads the same flat entry (and the same term, bit for bit).
__device__ __forceinline__ float bin_sat(float d, const Tab<float>& tb) {
  return __saturatef(fmaf(d, tb.k1, tb.k2));
}

// The term at bin coordinate us, its entry fetched through the texture path
// only where `need` is nonzero; elsewhere nothing is read and the result is
// 0.  The fetch is predicated rather than branched around, so a warp whose
// lanes disagree keeps its loads in flight together and the texture unit
// only serves the lanes that read.
__device__ __forceinline__ float term_tex_if(int row_e, float us, const Tab<float>& tb,
                                             unsigned need) {
  const float f = __fmaf_rd(us, tb.umax, 8388608.0f);
  const int e = row_e - 0x4B000000 + __float_as_int(f);
  float x = 0.f, y = 0.f, z = 0.f, w = 0.f;
  asm("{\n\t.reg .pred q;\n\tsetp.ne.u32 q, %5, 0;\n\t"
      "@q tex.1d.v4.f32.s32 {%0, %1, %2, %3}, [%4, {%6}];\n\t}"
      : "+f"(x), "+f"(y), "+f"(z), "+f"(w)
      : "l"((unsigned long long)tb.tex), "r"(need), "r"(e));
  return fmaf(us, y, x);
}

// The same through L1 loads from the row's address.
__device__ __forceinline__ float term_ldg_if(const float2* __restrict__ row, float us,
                                             const Tab<float>& tb, unsigned need) {
  const float f = __fmaf_rd(us, tb.umax, 8388608.0f);
  const char* base = reinterpret_cast<const char*>(row) - 8ull * 0x4B000000u;
  float x = 0.f, y = 0.f;
  asm("{\n\t.reg .pred q;\n\t.reg .u64 ad;\n\tsetp.ne.u32 q, %3, 0;\n\t"
      "mad.wide.u32 ad, %2, 8, %4;\n\t"
      "@q ld.global.nc.v2.f32 {%0, %1}, [ad];\n\t}"
      : "+f"(x), "+f"(y)
      : "r"((unsigned)__float_as_int(f)), "r"(need), "l"(base));
  return fmaf(us, y, x);
}

// The same term read from a row staged in shared memory (32-bit address:
// one multiply-add forms the entry address).
__device__ __forceinline__ float pair_term_smem(uint32_t row, float d, const Tab<float>& tb) {
  const float us = __saturatef(fmaf(d, tb.k1, tb.k2));
  const float f = __fmaf_rd(us, tb.umax, 8388608.0f);
  const uint32_t ad = row - 8u * 0x4B000000u + 8u * (uint32_t)__float_as_int(f);
  float2 v;
  asm volatile("ld.shared.v2.f32 {%0, %1}, [%2];" : "=f"(v.x), "=f"(v.y) : "r"(ad));
  return fmaf(us, v.y, v.x);
}

// ------------------------------------------------------------------ async copies
__device__ __forceinline__ uint32_t smem_addr(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ void mbar_init(uint32_t bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_init_fence() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint32_t bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes)
               : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint32_t bar, unsigned parity) {
  unsigned ok;
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
      "selp.u32 %0, 1, 0, p;\n\t}"
      : "=r"(ok)
      : "r"(bar), "r"(parity)
      : "memory");
  return ok != 0;
}
// Bounded wait for phase `parity` of an mbarrier: gives up (false) after
// 2^24 tries or about 2^31 clock cycles (~1 s), whichever comes first.
__device__ __forceinline__ bool mbar_wait_bounded(uint32_t bar, unsigned parity) {
  if (mbar_try_wait(bar, parity)) return true;
  const long long t0 = clock64();
  for (int i = 0; i < (1 << 24); ++i) {
    if (mbar_try_wait(bar, parity)) return true;
    if (clock64() - t0 > (1ll << 31)) break;
  }
  return false;
}
// Wait for phase `parity` of an mbarrier with at most `tries` polls (the
// staging ring's test hook: a wait that is meant to give up).
__device__ __forceinline__ bool mbar_wait_tries(uint32_t bar, unsigned parity, int tries) {
  for (int i = 0; i < tries; ++i)
    if (mbar_try_wait(bar, parity)) return true;
  return false;
}
// Order this thread's earlier generic-proxy accesses of shared memory before
// later async-proxy (bulk copy) writes to it.
__device__ __forceinline__ void fence_proxy_async_smem() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
// Bulk copy of `bytes` (multiple of 16, both ends 16-byte aligned) from
// global to this CTA's shared memory, completing on mbarrier `bar`.
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, unsigned bytes,
                                         uint32_t bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::
          "r"(dst),
      "l"(src), "r"(bytes), "r"(bar)
      : "memory");
}

// Row r(a,b) = a L - a(a+1)/2 + (b-a-1), a < b.
__device__ __forceinline__ int row_of(int L, int a, int b) {
  return a * L - ((a * (a + 1)) >> 1) + (b - a - 1);
}

// ------------------------------------------------------------------ RNG
// Philox4x32-10: ten rounds of two 32x32->64 products by fixed odd
// multipliers, XOR with the other words and the round key, word swap; the
// key advances by fixed Weyl constants between rounds.
__device__ __forceinline__ uint4 philox4x32_10(uint4 x, uint2 k) {
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    if (r) {
      k.x += 0x9E3779B9u;
      k.y += 0xBB67AE85u;
    }
    const uint32_t a_lo = 0xD2511F53u * x.x, a_hi = __umulhi(0xD2511F53u, x.x);
    const uint32_t b_lo = 0xCD9E8D57u * x.z, b_hi = __umulhi(0xCD9E8D57u, x.z);
    x = make_uint4(b_hi ^ x.y ^ k.x, b_lo, a_hi ^ x.w ^ k.y, a_lo);
  }
  return x;
}

__device__ __forceinline__ uint4 draw_words(unsigned long long seed, uint32_t chain,
                                            unsigned long long t, uint32_t stream) {
  return philox4x32_10(make_uint4(chain, (uint32_t)t, (uint32_t)(t >> 32), stream),
                       make_uint2((uint32_t)seed, (uint32_t)(seed >> 32)));
}

// ((w >> 9) + 1/2) / 2^23: exact in binary32.
__device__ __forceinline__ float uniform23f(uint32_t w) {
  return (float)((w >> 9)) * 0x1p-23f + 0x1p-24f;
}
__device__ __forceinline__ double uniform23d(uint32_t w) {
  return (double)((w >> 9)) * 0x1p-23 + 0x1p-24;
}

// Box-Muller normal z and ln u for one proposal, in precision R.
__device__ __forceinline__ void normal_and_lnu(uint4 w, float* z, float* lnu) {
  float u0 = uniform23f(w.x), u1 = uniform23f(w.y), u2 = uniform23f(w.z);
  *z = sqrtf(-2.0f * logf(u0)) * cospif(2.0f * u1);
  *lnu = logf(u2);
}
__device__ __forceinline__ void normal_and_lnu(uint4 w, double* z, double* lnu) {
  double u0 = uniform23d(w.x), u1 = uniform23d(w.y), u2 = uniform23d(w.z);
  *z = sqrt(-2.0 * log(u0)) * cospi(2.0 * u1);
  *lnu = log(u2);
}

template <class R>
__device__ __forceinline__ R pi_() {
  return R(3.14159265358979323846);
}

// Wrap to (-pi, pi].
template <class R>
__device__ __forceinline__ R wrap_angle(R a) {
  const R tp = R(2) * pi_<R>();
  R w = a - tp * floor(a / tp + R(0.5));
  if (w <= -pi_<R>()) w += tp;
  if (w > pi_<R>()) w -= tp;
  return w;
}
// FP32: the turn count from a product with 1/(2 pi) (one multiply, no
// division); a count off by one at the ends is set right by the checks.
template <>
__device__ __forceinline__ float wrap_angle<float>(float a) {
  const float tp = 2.f * pi_<float>();
  float w = a - tp * floorf(fmaf(a, 0.15915494309189535f, 0.5f));
  if (w <= -pi_<float>()) w += tp;
  if (w > pi_<float>()) w -= tp;
  return w;
}

// Proposed torsion for current value th, normal z and step sigma; lattice
// mode snaps to multiples of q = 2 pi / K.
template <class R>
__device__ __forceinline__ R propose(R th, R z, R sigma, int lattice_K) {
  R prop = th + sigma * z;
  if (lattice_K > 0) {
    const R q = R(2) * pi_<R>() / R(lattice_K);
    prop = q * rint(prop / q);
  }
  return wrap_angle(prop);
}

// ------------------------------------------------------------------ trace
struct TraceRec {
  int k;
  int accept;
  double theta_new;
  double lnu;
  double dE;
};

// ------------------------------------------------------------------ problem tables
struct ProteinDev {
  int L, n;
  long long tab_off;  // element offset of row 0 of this protein's table
  int chain0;         // first chain id of this protein
  int nchains;
  long long tors0;    // element offset of chain0's torsions
};

struct GroupDev {
  int protein;
  int chain0;   // absolute id of the group's first chain
  int nchains;  // chains in this group (<= chains per CTA)
  int pad;
};

// Allow a kernel to use all dynamic shared memory the device offers on top of
// its static shared memory.
template <class K>
inline cudaError_t allow_dynamic_smem(K kernel, size_t optin) {
  cudaFuncAttributes at;
  cudaError_t e = cudaFuncGetAttributes(&at, kernel);
  if (e != cudaSuccess) return e;
  const size_t stat = at.sharedSizeBytes;
  const size_t dyn = optin > stat ? optin - stat : 0;
  return cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

}  // namespace amh
