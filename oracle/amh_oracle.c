/*
 * amh_oracle.c -- plain, slow, FP64 CPU oracle for the Alternating
 * Metropolis-Hastings (AMH) hot path of Ghantasala, Jaiswal & Datta,
 * "An Efficient MCMC Approach to Energy Function Optimization in Protein
 * Structure Prediction" (arXiv 2211.03193).
 *
 * TEST INFRASTRUCTURE ONLY.  Only the test suite, the smoke check and the
 * benchmark's CPU-baseline leg load this file.  It shares no code, header,
 * constant table or helper with the CUDA library: every formula here is
 * written out again from the paper and the published methods it names.
 *
 * What it computes, in the paper's order and notation:
 *   - G(s): torsions -> backbone N, CA, C and virtual C-beta coordinates
 *     (Sec. 2.1 / Eq. 3 text "x = G(s)"; the paper names no construction,
 *     so the Natural Extension Reference Frame placement of Parsons et al.,
 *     J. Comput. Chem. 26 (2005) 1063, is used with ideal geometry).
 *   - V(x): distogram energy, Eq. 5, summed over unordered pairs a<b, each
 *     term -ln p linearly interpolated between bin centres.
 *   - V_local(x,k,d): Eq. 6, the same sum restricted to residues
 *     floor(k/2) -+ floor(d/2), clipped to the chain.
 *   - Proposal: single-flip Gaussian step on one torsion (Eq. 2, Alg. 1),
 *     Metropolis test (Eq. 1, Eq. 3; acceptance ratio read as
 *     exp(-(V' - V)/T)), global sweeps use V, local sweeps use V_local.
 *   - Random numbers: Philox4x32-10 (Salmon, Moraes, Dror & Shaw, SC'11)
 *     and Box-Muller, standing in for the per-block LFSRs of Sec. 2.4.
 *   - dV/ds by the chain rule (for the gradient hand-off to L-BFGS named
 *     in the abstract).
 *
 * Every global proposal recomputes V(G(s')) over ALL pairs and compares it
 * with the cached V(G(s)); every local proposal recomputes V_local on both
 * states.  Nothing is blocked, fused or reordered.
 *
 * Build: gcc -O2 -ffp-contract=off -fopenmp -fPIC -shared (OpenMP is used
 * only to run independent chains side by side).
 */
#include <math.h>
#include <stdint.h>
#include <stdlib.h>
#include <string.h>

#ifdef _OPENMP
#include <omp.h>
#endif

/* ------------------------------------------------------------------ */
/* Ideal geometry.  The paper fixes none of these values (Sec. 2.3 only
 * says x = G(phi, psi)).  Bond lengths N-CA 1.458, CA-C 1.525, C-N 1.329 A
 * are the benchmark problem's; bond angles are the Engh & Huber (1991)
 * ideal values; omega = 180 deg; the virtual C-beta uses bond 1.52 A,
 * angle C-CA-CB 109.5 deg and improper dihedral N-C-CA-CB +122.6 deg
 * (L-chirality).                                                       */
#define ORC_PI 3.14159265358979323846
static const double B_N_CA = 1.458, B_CA_C = 1.525, B_C_N = 1.329;
static const double A_N_CA_C = 111.2, A_CA_C_N = 116.2, A_C_N_CA = 121.7;
static const double OMEGA_DEG = 180.0;
static const double B_CA_CB = 1.52, A_C_CA_CB = 109.5, T_N_C_CA_CB = 122.6;

static double deg2rad(double d) { return d * ORC_PI / 180.0; }

typedef struct { double x, y, z; } v3;
static v3 vsub(v3 a, v3 b) { v3 r = {a.x - b.x, a.y - b.y, a.z - b.z}; return r; }
static v3 vadd(v3 a, v3 b) { v3 r = {a.x + b.x, a.y + b.y, a.z + b.z}; return r; }
static v3 vscale(v3 a, double s) { v3 r = {a.x * s, a.y * s, a.z * s}; return r; }
static double vdot(v3 a, v3 b) { return a.x * b.x + a.y * b.y + a.z * b.z; }
static v3 vcross(v3 a, v3 b) {
  v3 r = {a.y * b.z - a.z * b.y, a.z * b.x - a.x * b.z, a.x * b.y - a.y * b.x};
  return r;
}
static double vnorm(v3 a) { return sqrt(vdot(a, a)); }
static v3 vunit(v3 a) { return vscale(a, 1.0 / vnorm(a)); }

/* NeRF placement (Parsons et al. 2005): the atom D bonded to C with
 * |CD| = bond, angle B-C-D = angle, dihedral A-B-C-D = torsion.         */
static v3 nerf_place(v3 A, v3 B, v3 C, double bond, double angle, double torsion) {
  v3 bc = vunit(vsub(C, B));
  v3 n = vunit(vcross(vsub(B, A), bc));
  v3 m = vcross(n, bc);
  double dx = -bond * cos(angle);
  double dy = bond * sin(angle) * cos(torsion);
  double dz = bond * sin(angle) * sin(torsion);
  return vadd(C, vadd(vscale(bc, dx), vadd(vscale(m, dy), vscale(n, dz))));
}

/* G(s): s[2i] = phi_i, s[2i+1] = psi_i (Sec. 2.1, Fig. 2 caption).
 * Output arrays are [L][3] row-major.  phi_0 and psi_{L-1} have no atom
 * to place and therefore no effect.                                     */
void orc_build(int L, const double* s, double* N, double* CA, double* C, double* CB) {
  v3* n = (v3*)malloc(sizeof(v3) * (size_t)L);
  v3* a = (v3*)malloc(sizeof(v3) * (size_t)L);
  v3* c = (v3*)malloc(sizeof(v3) * (size_t)L);
  const double aNCAC = deg2rad(A_N_CA_C), aCACN = deg2rad(A_CA_C_N), aCNCA = deg2rad(A_C_N_CA);
  n[0].x = 0; n[0].y = 0; n[0].z = 0;
  a[0].x = B_N_CA; a[0].y = 0; a[0].z = 0;
  c[0].x = B_N_CA - B_CA_C * cos(aNCAC); c[0].y = B_CA_C * sin(aNCAC); c[0].z = 0;
  for (int i = 0; i + 1 < L; ++i) {
    n[i + 1] = nerf_place(n[i], a[i], c[i], B_C_N, aCACN, s[2 * i + 1]);           /* psi_i   */
    a[i + 1] = nerf_place(a[i], c[i], n[i + 1], B_N_CA, aCNCA, deg2rad(OMEGA_DEG)); /* omega_i */
    c[i + 1] = nerf_place(c[i], n[i + 1], a[i + 1], B_CA_C, aNCAC, s[2 * (i + 1)]); /* phi_i+1 */
  }
  for (int i = 0; i < L; ++i) {
    v3 cb = nerf_place(n[i], c[i], a[i], B_CA_CB, deg2rad(A_C_CA_CB), deg2rad(T_N_C_CA_CB));
    if (N) { N[3 * i] = n[i].x; N[3 * i + 1] = n[i].y; N[3 * i + 2] = n[i].z; }
    if (CA) { CA[3 * i] = a[i].x; CA[3 * i + 1] = a[i].y; CA[3 * i + 2] = a[i].z; }
    if (C) { C[3 * i] = c[i].x; C[3 * i + 1] = c[i].y; C[3 * i + 2] = c[i].z; }
    if (CB) { CB[3 * i] = cb.x; CB[3 * i + 1] = cb.y; CB[3 * i + 2] = cb.z; }
  }
  free(n); free(a); free(c);
}

/* ------------------------------------------------------------------ */
/* Distogram table.  p[r][j] for the unordered pair r = r(a,b), a<b, with
 * r(a,b) = a*L - a(a+1)/2 + (b-a-1); bins j in ascending distance order,
 * edges[0..B] ascending, edges[B] may be +inf (overflow bin).
 * The energy term is -ln p (Eq. 5), interpolated linearly between bin
 * centres in -ln p (the reading of Eq. 5 used throughout: interpolating
 * the log keeps far bins finite where p underflows).  Centre of a finite
 * bin: midpoint of its edges; centre of an open last bin: its lower edge
 * plus half the width of the bin below it.  Below the first centre and
 * above the last centre the term is flat.  p is floored at 1e-300.     */
typedef struct {
  int L, B;
  double* E;       /* [rows][B] -ln p */
  double* centre;  /* [B] */
} orc_problem;

orc_problem* orc_problem_new(int L, int B, const double* p, const double* edges) {
  if (L < 1 || B < 2) return NULL;
  orc_problem* P = (orc_problem*)calloc(1, sizeof(orc_problem));
  size_t rows = (size_t)L * (size_t)(L - 1) / 2;
  P->L = L; P->B = B;
  P->E = (double*)malloc(sizeof(double) * (rows ? rows : 1) * (size_t)B);
  P->centre = (double*)malloc(sizeof(double) * (size_t)B);
  for (size_t i = 0; i < rows * (size_t)B; ++i) {
    double q = p[i] > 1e-300 ? p[i] : 1e-300;
    P->E[i] = -log(q);
  }
  for (int j = 0; j < B; ++j) {
    if (isinf(edges[j + 1]))
      P->centre[j] = edges[j] + 0.5 * (edges[j] - edges[j - 1]);
    else
      P->centre[j] = 0.5 * (edges[j] + edges[j + 1]);
  }
  return P;
}

void orc_problem_free(orc_problem* P) {
  if (!P) return;
  free(P->E); free(P->centre); free(P);
}

void orc_problem_centres(const orc_problem* P, double* out) {
  memcpy(out, P->centre, sizeof(double) * (size_t)P->B);
}

static size_t row_index(int L, int a, int b) {
  return (size_t)a * (size_t)L - (size_t)a * (size_t)(a + 1) / 2 + (size_t)(b - a - 1);
}

/* e_ab(d): piecewise-linear -ln p through (centre_j, E_j).  The segment
 * [c_j, c_{j+1}) is closed on the left.                                  */
double orc_pair_term(const orc_problem* P, int a, int b, double d) {
  const double* E = P->E + row_index(P->L, a, b) * (size_t)P->B;
  const double* c = P->centre;
  int B = P->B;
  if (d <= c[0]) return E[0];
  if (d >= c[B - 1]) return E[B - 1];
  int j = 0;
  while (!(d >= c[j] && d < c[j + 1])) ++j;
  double t = (d - c[j]) / (c[j + 1] - c[j]);
  return E[j] + t * (E[j + 1] - E[j]);
}

/* d e_ab / d d, the slope of the segment containing d (0 on flat ends). */
double orc_pair_slope(const orc_problem* P, int a, int b, double d) {
  const double* E = P->E + row_index(P->L, a, b) * (size_t)P->B;
  const double* c = P->centre;
  int B = P->B;
  if (d < c[0] || d >= c[B - 1]) return 0.0;
  int j = 0;
  while (!(d >= c[j] && d < c[j + 1])) ++j;
  return (E[j + 1] - E[j]) / (c[j + 1] - c[j]);
}

static double dist(const double* X, int a, int b) {
  double dx = X[3 * a] - X[3 * b], dy = X[3 * a + 1] - X[3 * b + 1], dz = X[3 * a + 2] - X[3 * b + 2];
  return sqrt(dx * dx + dy * dy + dz * dz);
}

/* Eq. 5 over unordered pairs a<b of C-beta coordinates CB[L][3]. */
double orc_energy(const orc_problem* P, const double* CB) {
  double V = 0.0;
  for (int a = 0; a < P->L; ++a)
    for (int b = a + 1; b < P->L; ++b) V += orc_pair_term(P, a, b, dist(CB, a, b));
  return V;
}

/* Eq. 6: residues i,j in [floor(k/2) - floor(d/2), floor(k/2) + floor(d/2)],
 * inclusive, clipped to [0, L-1], i<j.                                   */
double orc_energy_local(const orc_problem* P, const double* CB, int k, int d) {
  int c = k / 2, h = d / 2;
  int lo = c - h < 0 ? 0 : c - h;
  int hi = c + h > P->L - 1 ? P->L - 1 : c + h;
  double V = 0.0;
  for (int a = lo; a <= hi; ++a)
    for (int b = a + 1; b <= hi; ++b) V += orc_pair_term(P, a, b, dist(CB, a, b));
  return V;
}

double orc_energy_of_torsions(const orc_problem* P, const double* s) {
  double* CB = (double*)malloc(sizeof(double) * 3 * (size_t)P->L);
  orc_build(P->L, s, NULL, NULL, NULL, CB);
  double V = orc_energy(P, CB);
  free(CB);
  return V;
}

/* ------------------------------------------------------------------ */
/* Philox4x32-10 (Salmon et al., SC'11): a 4-word counter is passed ten
 * times through a round made of two 32x32->64 multiplications by fixed
 * odd constants, XORs with the other two words and the round key, and a
 * word permutation; the 2-word key is advanced by fixed Weyl increments
 * between rounds.  Constants as published in that paper.               */
void orc_philox4x32_10(const uint32_t ctr_in[4], const uint32_t key_in[2], uint32_t out[4]) {
  const uint64_t MA = 0xD2511F53u, MB = 0xCD9E8D57u;
  const uint32_t WA = 0x9E3779B9u, WB = 0xBB67AE85u;
  uint32_t x0 = ctr_in[0], x1 = ctr_in[1], x2 = ctr_in[2], x3 = ctr_in[3];
  uint32_t k0 = key_in[0], k1 = key_in[1];
  for (int round = 0; round < 10; ++round) {
    if (round > 0) { k0 += WA; k1 += WB; }
    uint64_t pa = MA * (uint64_t)x0;
    uint64_t pb = MB * (uint64_t)x2;
    uint32_t pa_hi = (uint32_t)(pa >> 32), pa_lo = (uint32_t)pa;
    uint32_t pb_hi = (uint32_t)(pb >> 32), pb_lo = (uint32_t)pb;
    uint32_t y0 = pb_hi ^ x1 ^ k0;
    uint32_t y1 = pb_lo;
    uint32_t y2 = pa_hi ^ x3 ^ k1;
    uint32_t y3 = pa_lo;
    x0 = y0; x1 = y1; x2 = y2; x3 = y3;
  }
  out[0] = x0; out[1] = x1; out[2] = x2; out[3] = x3;
}

/* Counter layout: (chain, t_lo, t_hi, stream); key = (seed_lo, seed_hi).
 * stream 0: proposal of global proposal index t; stream 1: noisy restart
 * of torsion k (t = k).                                                  */
static void draw(uint64_t seed, uint32_t chain, uint64_t t, uint32_t stream, uint32_t out[4]) {
  uint32_t ctr[4] = {chain, (uint32_t)t, (uint32_t)(t >> 32), stream};
  uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
  orc_philox4x32_10(ctr, key, out);
}

/* A uniform on (0,1) from the top 23 bits of a word: ((w>>9)+1/2)/2^23.
 * Exactly representable in binary32 and binary64 (24 significant bits),
 * so a single-precision consumer sees the same value.                   */
static double uniform23(uint32_t w) { return ((double)(w >> 9) + 0.5) / 8388608.0; }

/* Box-Muller (first branch): z = sqrt(-2 ln u0) cos(2 pi u1). */
static double box_muller(uint32_t w0, uint32_t w1) {
  double u0 = uniform23(w0), u1 = uniform23(w1);
  return sqrt(-2.0 * log(u0)) * cos(2.0 * ORC_PI * u1);
}

void orc_draw(uint64_t seed, uint32_t chain, uint64_t t, uint32_t stream, uint32_t out[4],
              double* z, double* u) {
  draw(seed, chain, t, stream, out);
  if (z) *z = box_muller(out[0], out[1]);
  if (u) *u = uniform23(out[2]);
}

/* Wrap to (-pi, pi]. */
static double wrap_angle(double a) {
  double w = a - 2.0 * ORC_PI * floor(a / (2.0 * ORC_PI) + 0.5);
  if (w <= -ORC_PI) w += 2.0 * ORC_PI;
  if (w > ORC_PI) w -= 2.0 * ORC_PI;
  return w;
}

/* ------------------------------------------------------------------ */
/* One MCMC run for one chain.
 *
 * mode 1 (global, Alg. 1 first inner loop): proposal index t runs from t0
 * to t0+steps-1, torsion k = t mod n.  s'_k = s_k + sigma*z (Eq. 2), then
 * accept iff ln u < -(V(G(s')) - V(G(s)))/T (Eq. 1, Eq. 3).
 * mode 0 (local, Alg. 1 second inner loop, Eqs. 4a-b, Eq. 6): whole
 * sweeps only (t0 and steps multiples of n).  The Metropolis test uses
 * V_local(G(s'),k,d) - V_local(G(s),k,d).  Within a sweep the torsions are
 * visited by colour: every k with k = r (mod max(4*floor(d/2),1)) for
 * r = 0,1,..., ascending k within a colour.  The proposal of torsion k in
 * sweep q always uses Philox index t = q*n + k, whatever the visiting
 * order.
 *
 * lattice_K > 0 (test mode): s'_k = q*round((s_k + sigma*z)/q), q=2pi/K,
 * a symmetric proposal on a K-point lattice.
 *
 * trace (optional, [steps] records in visiting order): k, z, ln u, dV,
 * accept.  forced (optional, [steps]): when non-NULL the run adopts these
 * decisions instead of its own (teacher forcing); its own decision is
 * still written to trace_own.
 * Returns the number of accepted proposals, or -1 on bad arguments.     */
typedef struct {
  int32_t k;
  int32_t accept;
  double z;
  double lnu;
  double dV;
  double theta_new;
} orc_trace_rec;

long long orc_run(const orc_problem* P, int mode, int window, double T, double sigma,
                  long long t0, long long steps, uint64_t seed, uint32_t chain, int lattice_K,
                  double* s, orc_trace_rec* trace, const uint8_t* forced) {
  const int L = P->L, n = 2 * L;
  if (steps < 0 || t0 < 0 || !(T > 0)) return -1;
  if (mode == 0 && ((t0 % n) != 0 || (steps % n) != 0)) return -1;
  double* CB = (double*)malloc(sizeof(double) * 3 * (size_t)L);
  double* CBn = (double*)malloc(sizeof(double) * 3 * (size_t)L);
  double* sn = (double*)malloc(sizeof(double) * (size_t)n);
  memcpy(sn, s, sizeof(double) * (size_t)n);
  orc_build(L, s, NULL, NULL, NULL, CB);
  double V = (mode == 1) ? orc_energy(P, CB) : 0.0;
  const double q = lattice_K > 0 ? 2.0 * ORC_PI / lattice_K : 0.0;
  const int h = window / 2;
  const int ncol = 4 * h > 1 ? 4 * h : 1;
  long long acc = 0;
  for (long long j = 0; j < steps; ++j) {
    long long t;
    int k;
    if (mode == 1) {
      t = t0 + j;
      k = (int)(t % n);
    } else {
      long long sweep = (t0 + j) / n;
      int slot = (int)((t0 + j) % n);
      /* slot -> torsion in colour order */
      int r = 0, rem = slot;
      for (r = 0; r < ncol; ++r) {
        int cnt = r < n ? (n - 1 - r) / ncol + 1 : 0;
        if (rem < cnt) break;
        rem -= cnt;
      }
      k = r + rem * ncol;
      t = sweep * (long long)n + k;
    }
    uint32_t w[4];
    double z, u;
    orc_draw(seed, chain, (uint64_t)t, 0, w, &z, &u);
    double lnu = log(u);
    double prop = s[k] + sigma * z;
    if (lattice_K > 0) prop = q * nearbyint(prop / q);
    double snew = wrap_angle(prop);
    sn[k] = snew;
    orc_build(L, sn, NULL, NULL, NULL, CBn);
    double dV, Vn = 0.0;
    if (mode == 1) {
      Vn = orc_energy(P, CBn);
      dV = Vn - V;
    } else {
      dV = orc_energy_local(P, CBn, k, window) - orc_energy_local(P, CB, k, window);
    }
    int own = lnu < -dV / T;
    int take = forced ? (int)forced[j] : own;
    if (trace) {
      trace[j].k = k; trace[j].accept = own; trace[j].z = z; trace[j].lnu = lnu;
      trace[j].dV = dV; trace[j].theta_new = snew;
    }
    if (take) {
      s[k] = snew;
      memcpy(CB, CBn, sizeof(double) * 3 * (size_t)L);
      if (mode == 1) V = Vn;
      ++acc;
    } else {
      sn[k] = s[k];
    }
  }
  free(CB); free(CBn); free(sn);
  return acc;
}

/* Many chains of one problem side by side (independent; OpenMP only
 * distributes whole chains).  s: [nchains][n], chain ids chain0+c.      */
long long orc_run_chains(const orc_problem* P, int nchains, int mode, int window, double T,
                         double sigma, long long t0, long long steps, uint64_t seed,
                         uint32_t chain0, int lattice_K, double* s, long long* accepted) {
  const int n = 2 * P->L;
  long long total = 0;
  int bad = 0;
#pragma omp parallel for schedule(dynamic, 1) reduction(+ : total) reduction(| : bad)
  for (int c = 0; c < nchains; ++c) {
    long long a = orc_run(P, mode, window, T, sigma, t0, steps, seed, chain0 + (uint32_t)c,
                          lattice_K, s + (size_t)c * (size_t)n, NULL, NULL);
    if (a < 0) bad = 1;
    if (accepted) accepted[c] = a;
    total += a;
  }
  return bad ? -1 : total;
}

int orc_num_threads(void) {
#ifdef _OPENMP
  return omp_get_max_threads();
#else
  return 1;
#endif
}

/* Noisy restart: s_k += sd * z_k for every torsion, z_k from stream 1 at
 * index k, then wrap (the noisy-restart baseline of Sec. 3 with a
 * Gaussian kick).                                                        */
void orc_noisy_restart(int L, double* s, double sd, uint64_t seed, uint32_t chain) {
  for (int k = 0; k < 2 * L; ++k) {
    uint32_t w[4];
    double z;
    orc_draw(seed, chain, (uint64_t)k, 1, w, &z, NULL);
    s[k] = wrap_angle(s[k] + sd * z);
  }
}

/* ------------------------------------------------------------------ */
/* dV/ds_k by the chain rule.  Changing s_k rotates every atom on the far
 * side of its bond (Sec. 2.4, "Proposal Generation") about the bond axis:
 * phi_i about N_i->CA_i, moving CB_b for b >= i; psi_i about CA_i->C_i,
 * moving CB_b for b >= i+1.  For a moving CB_b, d x_b / d s_k =
 * u x (x_b - o) with u the unit bond axis and o a point on it, so
 * dV/ds_k = sum over pairs (a<p<=b) of e'_ab(d_ab) (x_b - x_a)/d_ab .
 * u x (x_b - o).  Pairs on the same side keep their distance.  Written
 * pair by pair for every k: O(n L^2), slow on purpose.                  */
void orc_grad(const orc_problem* P, const double* s, double* V_out, double* g) {
  const int L = P->L, n = 2 * L;
  double* N = (double*)malloc(sizeof(double) * 3 * (size_t)L);
  double* CA = (double*)malloc(sizeof(double) * 3 * (size_t)L);
  double* C = (double*)malloc(sizeof(double) * 3 * (size_t)L);
  double* CB = (double*)malloc(sizeof(double) * 3 * (size_t)L);
  orc_build(L, s, N, CA, C, CB);
  if (V_out) *V_out = orc_energy(P, CB);
  for (int k = 0; k < n; ++k) {
    int i = k / 2;
    v3 o, u;
    int p;
    if (k % 2 == 0) { /* phi_i */
      v3 An = {N[3 * i], N[3 * i + 1], N[3 * i + 2]};
      v3 Aca = {CA[3 * i], CA[3 * i + 1], CA[3 * i + 2]};
      o = An; u = vunit(vsub(Aca, An)); p = i;
    } else {          /* psi_i */
      v3 Aca = {CA[3 * i], CA[3 * i + 1], CA[3 * i + 2]};
      v3 Ac = {C[3 * i], C[3 * i + 1], C[3 * i + 2]};
      o = Aca; u = vunit(vsub(Ac, Aca)); p = i + 1;
    }
    double acc = 0.0;
    for (int a = 0; a < L && a < p; ++a) {
      for (int b = p; b < L; ++b) {
        if (b <= a) continue;
        double d = dist(CB, a, b);
        double sl = orc_pair_slope(P, a, b, d);
        if (sl == 0.0) continue;
        v3 xb = {CB[3 * b], CB[3 * b + 1], CB[3 * b + 2]};
        v3 xa = {CB[3 * a], CB[3 * a + 1], CB[3 * a + 2]};
        v3 dir = vscale(vsub(xb, xa), 1.0 / d);
        v3 vel = vcross(u, vsub(xb, o));
        acc += sl * vdot(dir, vel);
      }
    }
    g[k] = acc;
  }
  free(N); free(CA); free(C); free(CB);
}

/* ------------------------------------------------------------------ */
/* Replica exchange between neighbouring temperatures (parallel tempering,
 * one of the coordinated multi-chain schemes Sec. 2.4 lists for the
 * chains a GPU runs side by side; Hansmann 1997).  Chains are grouped in
 * ladders of K consecutive chains; slot j of a ladder runs at temperature
 * T_scale * ladder[j].  For every pair of slots (j, j+1) with j = parity
 * (mod 2), the states are swapped iff ln u < (1/T_j - 1/T_{j+1})(E_j - E_{j+1}),
 * u at Philox counter (chain of slot j, round low, round high, 3): the
 * Metropolis rule for exchanging two replicas of exp(-E/T) (u from Philox
 * stream 3).  E and the torsions s[nchains][n] are swapped together;
 * accepted[chain of slot j] is set to 1 for an exchange.                 */
void orc_exchange(int nchains, int n, int K, const double* ladder, double T_scale, int parity,
                  uint64_t seed, uint64_t round, uint32_t chain0, double* E, double* s,
                  int* accepted) {
  for (int c = 0; c < nchains; ++c) accepted[c] = 0;
  for (int base = 0; base + K <= nchains; base += K) {
    for (int j = parity; j + 1 < K; j += 2) {
      int a = base + j, b = base + j + 1;
      double Ta = T_scale * ladder[j], Tb = T_scale * ladder[j + 1];
      uint32_t w[4];
      uint32_t ctr[4] = {chain0 + (uint32_t)a, (uint32_t)round, (uint32_t)(round >> 32), 3u};
      uint32_t key[2] = {(uint32_t)seed, (uint32_t)(seed >> 32)};
      orc_philox4x32_10(ctr, key, w);
      double lnu = log(uniform23(w[0]));
      double delta = (1.0 / Ta - 1.0 / Tb) * (E[a] - E[b]);
      if (lnu < delta) {
        double t = E[a]; E[a] = E[b]; E[b] = t;
        for (int k = 0; k < n; ++k) {
          double q = s[(size_t)a * n + k];
          s[(size_t)a * n + k] = s[(size_t)b * n + k];
          s[(size_t)b * n + k] = q;
        }
        accepted[a] = 1;
      }
    }
  }
}
