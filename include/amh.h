/*
 * amh.h -- C ABI of the GB300 (sm_103a) Alternating Metropolis-Hastings
 * library: many independent MCMC chains over backbone torsions, scored by
 * a distogram energy (Ghantasala, Jaiswal & Datta, arXiv 2211.03193).
 *
 * Problem statement (Sec. 2.1, Sec. 2.3): the state of one chain is the
 * torsion vector s of n = 2L angles for a protein of L residues,
 * s[2i] = phi_i and s[2i+1] = psi_i (radians, wrapped to (-pi, pi]);
 * omega is fixed at 180 deg.  x = G(s) are the C-beta coordinates built by
 * NeRF with ideal geometry (N-CA 1.458, CA-C 1.525, C-N 1.329 A; N-CA-C
 * 111.2, CA-C-N 116.2, C-N-CA 121.7 deg; virtual C-beta 1.52 A, C-CA-CB
 * 109.5 deg, improper N-C-CA-CB +122.6 deg).  The energy is Eq. 5 over
 * unordered residue pairs a<b: V(x) = sum -ln p_ab(|x_a - x_b|), with -ln p
 * interpolated linearly between bin centres and flat beyond the first and
 * last centres; the window energy V_local(x,k,d) of Eq. 6 sums the pairs
 * inside residues floor(k/2) -+ floor(d/2).
 *
 * Conventions for every call:
 *  - Every call returns an amh_status; nothing throws across the ABI.
 *  - A context owns all of its device memory; the caller owns every buffer
 *    it passes in.  Inputs are copied; output buffers are written.
 *  - "host or device" pointers are told apart with cudaPointerGetAttributes;
 *    device pointers must be on the context's device.
 *  - All work is issued on the context's stream (amh_options.stream).
 *    Calls whose output is host memory synchronise that stream; calls
 *    whose outputs are device memory (or NULL) return without waiting.
 *  - A CUDA error or a bounded device wait that gave up makes the context
 *    sticky-broken: that call returns AMH_ECUDA (or AMH_ETIMEOUT) and every
 *    later call AMH_ESTATE until amh_destroy.
 *  - A context is used from one host thread at a time.
 */
#ifndef AMH_H
#define AMH_H

#ifdef __cplusplus
extern "C" {
#endif

typedef struct amh_ctx amh_ctx;

typedef enum {
  AMH_OK = 0,
  AMH_EINVAL = 1,   /* bad argument; nothing was done */
  AMH_ENOMEM = 2,   /* device allocation failed */
  AMH_ECUDA = 3,    /* CUDA runtime error (context is now broken) */
  AMH_ETIMEOUT = 4, /* a bounded device wait (shared-memory staging) gave up */
  AMH_ESTATE = 5    /* context broken by an earlier error, or NULL */
} amh_status;

typedef enum {
  AMH_LOCAL = 0,  /* localized MH: Eqs. 4a-b with V_local of Eq. 6 */
  AMH_GLOBAL = 1  /* traditional MH: Eqs. 1-3 with V of Eq. 5 */
} amh_mode;

typedef struct {
  int precision;           /* 32 (default): FP32 coordinates and pair terms,
                              energies summed in FP64; 64: FP64 throughout. */
  int resync_every;        /* global sweeps rebuild G(s) in FP64 from the
                              torsions every this many proposals (default
                              1000), at entry and at each new sweep; V is
                              recomputed from scratch when a call ends. */
  int chains_per_cta;      /* chains that share one CTA in global sweeps:
                              0 = autotuned at first use, else 1, 2, 4 or 8. */
  int threads_per_cta;     /* global sweeps: 0 = autotuned with chains_per_cta
                              (256 if chains_per_cta is set), else 64, 128,
                              256 or 512. */
  int trace_chains;        /* record every proposal of chains [0, trace_chains) */
  long long trace_capacity;/* records kept per traced chain (visit order) */
  int lattice_K;           /* test mode: 0 = off; K > 0 snaps proposals to a
                              K-point lattice, s' = q round((s + sigma z)/q),
                              q = 2 pi / K (symmetric proposal). */
  int table_is_neglog;     /* 0: table holds p; 1: table already holds -ln p */
  int stage_table;         /* global sweeps read the straddle block's table rows
                              0: as tuned (staged in shared memory by bulk
                              async copies when the autotuner finds it faster;
                              with a fixed chains_per_cta, staged when it fits
                              and the far-field skip is off), 1: always staged
                              (AMH_EINVAL if impossible: needs precision 32
                              and 4 or 8 chains per CTA), 2: never staged
                              (read through the L1 cache). */
  int table_texture;       /* precision 32, global sweeps: 0 = fetch table entries
                              through a 1-D texture (32-bit indices) when the
                              table fits the device's 1-D texture limit, else
                              global loads (default); 1 = texture (AMH_EINVAL if
                              it does not fit); 2 = global loads. */
  int far_pairs;           /* precision 32, global sweeps: 0 = skip the straddle
                              pairs that stay beyond the last bin centre before
                              and after the move (their Eq. 5 terms are equal,
                              so Delta V is unchanged; found per 12-atom chunk
                              of the fixed side by bounding spheres) (default);
                              1 = evaluate every straddle pair. */
  int local_chains_per_cta; /* local sweeps: chains per CTA, 0 (chosen from the
                              window: as many as keep one colour's windows
                              within 256 threads) or 1, 2, 4, 8, 16, 32 */
  int local_threads;       /* local sweeps: threads per CTA, 0 (256, fewer if
                              shared memory is short) or a multiple of 32 up
                              to 256; AMH_EINVAL at the sweep if the shape
                              does not fit in shared memory */
  void* stream;            /* cudaStream_t; NULL = the legacy default stream */
  int keep_coords;         /* 1: keep every chain's C-beta coordinates for
                              amh_get_coords (one buffer of 3 L values per
                              chain, written by global sweeps and energy
                              computations); 0 (default): not kept */
  int wait_test;           /* test hook of the bounded waits (0 = off, the
                              default).  N > 0: every CTA of a staged global
                              sweep first waits on its staging ring's first
                              slot before issuing any copy, giving up after N
                              tries.  Nothing can arrive there, so the wait
                              gives up with no copy in flight and the call
                              fails with AMH_ETIMEOUT. */
  int global_kernel;       /* global sweeps: 0 = chosen by the autotuner among
                              both kernels (the CTA kernel if chains_per_cta is
                              set); 1 = the CTA kernel (chains_per_cta chains
                              of a CTA in lock-step); 2 = chain groups: each
                              chain on warps_per_chain warps of its own, which
                              meet at their own barrier (chains_per_cta chains
                              per CTA: 0 = tuned, 1, 2, 4 or 8, at most 8
                              warps per CTA), which needs precision 32, the
                              far-field skip (far_pairs 0, L <= 768) and no
                              staging, else AMH_EINVAL.  Both kernels compute
                              the same proposals and decisions. */
  int warps_per_chain;     /* chain groups: 0 = tuned (1 with a fixed
                              chains_per_cta), 1, 2 or 4 */
} amh_options;

/* One proposal record (traced chains only), 32 bytes. */
typedef struct {
  int k;             /* torsion index */
  int accept;        /* 1 if accepted */
  double theta_new;  /* proposed value s'_k (radians, wrapped) */
  double lnu;        /* ln u of the accept uniform */
  double dE;         /* Delta V (global) or Delta V_local (local) used */
} amh_trace_rec;

/* Fill *opt with the defaults listed above. */
void amh_options_default(amh_options* opt);

/*
 * amh_init -- create a context holding n_proteins problems and their chains
 * (Alg. 1 "input": the initial state s^0 of every chain; Eq. 5's
 * distogram P(d | S, MSA(S)) per protein).
 *   L[p]                residues of protein p (2 <= L <= 4096)
 *   chains_per_protein  chains of protein p (>= 1); chain ids run protein
 *                       by protein: protein 0's chains first.
 *   torsions            host, float32, the chains' starting s concatenated
 *                       chain by chain: sum_p chains[p] * 2 L[p] values.
 *   table               host, float64, per protein in order, rows
 *                       r(a,b) = a L - a(a+1)/2 + (b-a-1) for a<b, each row
 *                       B values in ascending distance order: p (or -ln p
 *                       if table_is_neglog).  p is floored at 1e-300.
 *   edges               host, float64 [B+1] ascending, shared by all
 *                       proteins; edges[B] may be +INFINITY (open last bin,
 *                       centre = edges[B-1] + (edges[B-1]-edges[B-2])/2).
 *                       Bin centres must be evenly spaced (relative 1e-9),
 *                       else AMH_EINVAL.
 *   B                   bins, 2 <= B <= 256.
 *   opt                 options (NULL = defaults).
 * Computes G(s) and V for every chain; best energy = starting energy.
 */
amh_status amh_init(amh_ctx** out, int n_proteins, const int* L, const int* chains_per_protein,
                    const float* torsions, const double* table, const double* edges, int B,
                    const amh_options* opt);

/*
 * amh_energy -- V(G(s)) of Eq. 5 for every chain's current state: FP32 (or
 * FP64) pair terms summed in FP64.  E_out: [total chains] doubles, host or
 * device.
 */
amh_status amh_energy(amh_ctx* ctx, double* E_out);

/*
 * amh_sweep -- run `steps` Metropolis proposals on every chain (Alg. 1 inner
 * loops).  Each chain keeps a proposal counter t (0 after amh_init); the
 * proposal with index t perturbs torsion k = t mod n by sigma_rad * z
 * (Eq. 2), z and the accept uniform u drawn from Philox4x32-10 with key
 * `seed` and counter (chain id, t low word, t high word, 0); Box-Muller
 * z = sqrt(-2 ln u0) cos(2 pi u1) with u_i = ((w_i >> 9) + 1/2) / 2^23.
 * Accept iff ln u < -dE / T (Eq. 1 with P = exp(-V/T)).
 *   mode AMH_GLOBAL  dE = V(G(s')) - V(G(s)), k visited in order; window
 *                    ignored.
 *   mode AMH_LOCAL   dE = V_local(G(s'),k,d) - V_local(G(s),k,d), d = window
 *                    (0 <= d <= 64); whole sweeps only: t and steps must be
 *                    multiples of n for every protein, else AMH_EINVAL.
 *                    Within a sweep, torsions are visited by colour
 *                    (k mod max(4 floor(d/2), 1) ascending, then k
 *                    ascending); same-colour windows touch disjoint torsions
 *                    and are evaluated concurrently.
 *   accepted_out     NULL, or [total chains] long long (host or device):
 *                    accepted proposals of this call per chain.
 * Global sweeps end with V recomputed from scratch (FP32 terms of the current
 * coordinates, FP64 sum; FP64 form: G(s) rebuilt first) and update each
 * chain's best state.
 * Split calls equal one long call (the counter continues).
 */
amh_status amh_sweep(amh_ctx* ctx, int mode, int window, double T, double sigma_rad,
                     long long steps, unsigned long long seed, long long* accepted_out);

/*
 * amh_sweeps -- like amh_sweep but in whole sweeps: every chain of protein
 * p runs nsweeps * 2 L[p] proposals (for contexts holding proteins of
 * different lengths).
 */
amh_status amh_sweeps(amh_ctx* ctx, int mode, int window, double T, double sigma_rad,
                      long long nsweeps, unsigned long long seed, long long* accepted_out);

/*
 * amh_grad -- energy and its gradient for a batch of torsion vectors of one
 * protein of the context (the dV/ds the abstract's L-BFGS pairing needs).
 *   theta       device, [batch][2 L] (float32, or float64 if precision 64)
 *   E_out       device, [batch] doubles: V(G(theta))
 *   dE_dtheta   device, [batch][2 L], same type as theta
 * dV/ds_k = u_k . (M_p - o_k x G_p): G_p and M_p are suffix sums over C-beta
 * b >= p(k) of the pair-force sum g_b and of x_b x g_b; u_k the unit bond
 * axis and o_k its first atom.  Kinks of the piecewise-linear term take the
 * slope of the segment to their right.
 */
amh_status amh_grad(amh_ctx* ctx, int protein, const void* theta, int batch, double* E_out,
                    void* dE_dtheta);

/*
 * amh_sweeps_sched -- a run of nsweeps whole sweeps in one call (Alg. 1's
 * inner loop of N_local localized or N_global global sweeps), sweep q of the
 * run at temperature T[q] and step sigma_rad[q] (the annealing schedule of
 * Sec. 2.3 / Sec. 3 changes them from sweep to sweep).
 *   T, sigma_rad   host, [nsweeps] doubles; T[q] > 0.
 *   1 <= nsweeps <= AMH_MAX_SCHED; every chain's proposal counter must sit
 *   at a sweep boundary (t a multiple of n), else AMH_EINVAL.
 * The result equals nsweeps calls of amh_sweeps(.., 1, ..) with those T and
 * sigma (the same proposals, draws and decisions); accepted_out sums the run.
 */
#define AMH_MAX_SCHED 16
amh_status amh_sweeps_sched(amh_ctx* ctx, int mode, int window, int nsweeps, const double* T,
                            const double* sigma_rad, unsigned long long seed,
                            long long* accepted_out);

/*
 * amh_get_state -- copy out the chains' state; any pointer may be NULL.
 *   torsions_out, best_torsions  [sum chains * 2 L] float32 (host or device)
 *   E_out      V as of the last global sweep or amh_energy call [chains];
 *              after amh_set_state / amh_noisy_restart (with no global
 *              sweep since) V of the current state, computed by this call
 *   best_E     lowest energy seen at a global-sweep end [chains]
 */
amh_status amh_get_state(amh_ctx* ctx, float* torsions_out, double* E_out, double* best_E,
                         float* best_torsions);

/* amh_set_state -- replace every chain's torsions (host or device, float32,
 * layout as in amh_init; a host buffer may be reused when the call returns).
 * V is recomputed when next read (amh_get_state, amh_exchange), unless a
 * global sweep, which ends with V from scratch, comes first.  Counters and
 * best are kept.                                                            */
amh_status amh_set_state(amh_ctx* ctx, const float* torsions);

/* amh_noisy_restart -- s_k += sd_rad * z for every torsion of every chain,
 * z from Philox counter (chain, k, 0, 1) under key `seed`, then wrap; V is
 * recomputed as after amh_set_state (the noisy-restart baseline of Sec. 3). */
amh_status amh_noisy_restart(amh_ctx* ctx, double sd_rad, unsigned long long seed);

/*
 * amh_set_ladder -- parallel tempering (one of the coordinated multi-chain
 * schemes Sec. 2.4 names for chains run side by side): the chains of every
 * protein form ladders of K consecutive chains, and slot j of a ladder
 * runs its sweeps at T * ladder[j] (T the sweep call's temperature, so an
 * anneal scales the whole ladder).  Every protein's chain count must be a
 * multiple of K.  K = 0 removes the ladder.  ladder: host, K positive
 * factors, ascending for the usual ordering.
 */
amh_status amh_set_ladder(amh_ctx* ctx, int K, const double* ladder);

/*
 * amh_exchange -- one round of replica exchange: for every ladder slot j
 * with j = parity (mod 2) and j+1 < K, the states of slots j and j+1 are
 * swapped iff ln u < (1/T_j - 1/T_{j+1}) (E_j - E_{j+1}) with T_j = T *
 * ladder[j] (the Metropolis rule for exchanging two replicas), u from
 * Philox4x32-10 at counter (chain of slot j, round low, round high, 3)
 * where round counts this context's exchange calls.  Uses the stored
 * energies (recomputed first if the state was replaced since the last global
 * sweep or amh_energy): call it after a global sweep.  swapped_out: NULL
 * or [total chains] long long (host or device), 1 at the lower slot of each
 * swapped pair.
 */
amh_status amh_exchange(amh_ctx* ctx, double T, int parity, unsigned long long seed,
                        long long* swapped_out);

/* amh_get_trace -- copy the trace of chain `chain` (< trace_chains):
 * records [0, min(count, trace_capacity)) in visit order into `out` (host),
 * *count set to the records written so far.                              */
amh_status amh_get_trace(amh_ctx* ctx, int chain, amh_trace_rec* out, long long* count);

/* amh_counter -- the proposal counter t of chain `chain`. */
amh_status amh_counter(amh_ctx* ctx, int chain, long long* t);

/*
 * amh_pair_terms -- straddle-pair terms of the global sweeps of this context
 * so far (Sec. 2.4 scores every pair of the block a < p(k) <= b; each term is
 * e(|x_a - x_b|) at one configuration: the current one or a proposal's).
 *   *evaluated: terms whose table entry was read and interpolated;
 *   *formed (may be NULL): terms whose distance was formed, i.e. the
 *   evaluated ones plus, in the FP32 form, those of pairs found to lie at or
 *   past the last bin centre in every configuration (flat: they add exactly
 *   zero, so their entries are not read).
 * With far_pairs = 0 the pairs that whole chunk tests place beyond the last
 * bin centre are skipped before any distance is formed and counted in
 * neither.  Host pointers; cumulative since amh_init; synchronises the
 * context's stream.  AMH_EINVAL if evaluated is NULL.
 */
amh_status amh_pair_terms(amh_ctx* ctx, unsigned long long* evaluated,
                          unsigned long long* formed);

/*
 * amh_philox -- the sampler's random stream, for checking: for
 * t = t0 .. t0+count-1 writes Philox4x32-10(key seed; counter (chain,
 * t_lo, t_hi, stream)) to words_out[count][4] and, for stream 0, the FP32
 * Box-Muller normal and accept uniform to z_out/u_out (any may be NULL).
 * All output pointers are host memory.  Runs on the current device.
 */
amh_status amh_philox(unsigned long long seed, unsigned chain, unsigned long long t0,
                      unsigned stream, long long count, unsigned* words_out, float* z_out,
                      float* u_out);

/*
 * amh_get_coords -- the C-beta coordinates x = G(s) the context holds
 * (Sec. 2.1: x = G(s) defines the coordinates of all C-beta atoms), for
 * checking the builder and the moves against an independent G(s).  Needs
 * keep_coords = 1 at amh_init, else AMH_EINVAL.
 *   cb_out  host, double [sum over chains of L_p][3], chain by chain.
 * The coordinates are those of the last global sweep or energy computation
 * (the ones its V was summed from), widened from the context's precision:
 * after a global sweep, the coordinates the sweep ended with (rebuilt at
 * its last resync and moved rigidly by every accepted proposal since; a
 * rigid motion of the whole chain does not change V, and each move turns
 * the side of the pivot with fewer residues, so the frame is the chain's
 * own); after amh_init, amh_energy, or a state change read back,
 * G(s) built from the torsions in the canonical frame of residue 0 (N at the
 * origin, CA on +x, C in the xy-plane with y > 0).  Synchronises the stream.
 */
amh_status amh_get_coords(amh_ctx* ctx, double* cb_out);

/*
 * amh_window_coords -- the window coordinates a local sweep scores proposal
 * k with (Eq. 6: residues floor(k/2) -+ floor(d/2), clipped to the chain),
 * built from chain `chain`'s current torsions by the local sweep kernel's
 * own window builder: residue r of [lo, hi] in the canonical frame of
 * residue lo (as in amh_get_coords).  0 <= window <= 64.
 *   cb_out  host, double [hi - lo + 1][3].
 *   lo_out, hi_out  host, the window's first and last residue (may be NULL).
 * Synchronises the stream.
 */
amh_status amh_window_coords(amh_ctx* ctx, int chain, int k, int window, double* cb_out,
                             int* lo_out, int* hi_out);

/* Text of the last error of ctx (or of the last context-free call). */
const char* amh_last_error(const amh_ctx* ctx);

/* Launch shape of the global sweeps (after tuning): chains per CTA, threads
 * per CTA, staging-ring depth (0 = table rows read through L1) and kernel
 * (1 = chains of a CTA in lock-step, 2 = chain groups, threads / (32 chains)
 * warps per chain); any pointer may be NULL. */
amh_status amh_launch_config(amh_ctx* ctx, int* chains_per_cta, int* threads_per_cta,
                             int* stage_depth, int* kernel);

/* Free everything the context owns.  NULL is ignored. */
void amh_destroy(amh_ctx* ctx);

/*
 * amh_grad_noalloc -- amh_grad without a context and without allocating.
 * (The paper has no counterpart: this is a deployment variant.)
 *
 * For callers that must not call cudaMalloc: hosts whose device memory
 * belongs to a pool or caching allocator they do not control (a framework
 * that reserves the GPU's memory up front leaves nothing for a second
 * allocator, and allocating beside it fragments its pool), services that
 * run under a fixed device-memory budget decided at start-up (an allocation
 * later can fail in the middle of a run), and latency-bound loops that
 * cannot afford the device-wide synchronisation cudaMalloc and cudaFree may
 * imply.  amh_grad reads a
 * distogram table that amh_init prepared in device memory the library
 * allocated; here the table is prepared on every call into one static
 * device array of AMH_NOALLOC_MAX_ENTRIES (value, slope) entries of 8 bytes
 * (16 MiB; rows L(L-1)/2 times entries per row (B+1 rounded down to even)
 * must fit: L <= 332 for 37 bins), which every GPU that loads the library
 * holds until the process exits.  Larger problems return AMH_EINVAL.
 *   L, B, edges, table_is_neglog   as in amh_init (edges on the host)
 *   table       device, float64 [L(L-1)/2][B]: p (or -ln p)
 *   theta       device, float32 [batch][2 L]
 *   E_out       device, [batch] doubles;  dE_dtheta  device, float32 [batch][2 L]
 *   stream      cudaStream_t or NULL
 * FP32 pair terms as amh_grad at precision 32.  Runs asynchronously on
 * `stream`; no call allocates or frees memory.  The first call on each
 * device looks up the device address of the static array (with that device
 * current); make that first call before any stream capture.  All calls on a
 * device share the array and it keeps the last call's contents: calls that
 * overlap on the GPU (different streams, or different host threads) race and
 * must be serialised by the caller.  Errors: amh_last_error(NULL).
 */
#define AMH_NOALLOC_MAX_ENTRIES (1 << 21)
amh_status amh_grad_noalloc(int L, int B, const double* table, int table_is_neglog,
                            const double* edges, const float* theta, int batch, double* E_out,
                            float* dE_dtheta, void* stream);

#ifdef __cplusplus
}
#endif
#endif /* AMH_H */
