/*
 * sbci.h -- C ABI of the GB300 SBCI library (libsbci.so).
 *
 * SBCI (simulated-bifurcation-based configuration interaction, arXiv
 * 2603.06101) finds the lowest k eigenpairs of the FCI Hamiltonian H by
 * integrating a classical system whose positions are the CI coefficients
 * (Eq. 1-11, Algorithm 1).  Every step needs one H-product Z = H z (Eq. S9,
 * Eq. S32), the "sigma build", which this library runs as CUDA kernels for
 * sm_103a over alpha/beta determinant strings.
 *
 * Conventions shared by every entry point:
 *  - Orbitals are real; h1 is the n x n core Hamiltonian, eri the n^4
 *    chemists'-notation integrals (ij|kl), both row-major FP64.
 *  - A string is an m-subset of the n orbitals; strings are ordered by
 *    increasing bitmask value.  A determinant |Ia Ib> has all alpha creators
 *    (ascending) left of all beta creators (ascending).  CI vectors are FP64
 *    [Na][Nb] row-major with flat index Ia*Nb + Ib.
 *  - sigma is the electronic H c, without e_core; energies are totals
 *    (electronic + e_core).
 *  - The caller owns every pointer it passes.  Host arrays are read or
 *    written during the call only; the library keeps no caller pointer.
 *    "Device" pointers are CUDA global-memory addresses on the context's GPU.
 *  - Every call returns sbci_status; no exception crosses the ABI.  On an
 *    error, sbci_last_error() gives a thread-local message.
 *  - NaN/Inf in caller inputs -> SBCI_ERR_NUMERIC before any GPU work.
 *  - The library never traps or spins without bound on the GPU.
 *  - Size limits: 1 <= n <= 16, 0 <= nalpha, nbeta <= n, nalpha+nbeta >= 1.
 */
#ifndef SBCI_H
#define SBCI_H

#include <stddef.h>

#ifdef __cplusplus
extern "C" {
#endif

typedef struct sbci_ctx sbci_ctx;

typedef enum {
  SBCI_OK = 0,
  SBCI_ERR_INVALID = 1,       /* bad argument or call order */
  SBCI_ERR_NOMEM = 2,         /* device or host allocation failed */
  SBCI_ERR_CUDA = 3,          /* CUDA runtime error (message has the code) */
  SBCI_ERR_NUMERIC = 4,       /* NaN/Inf in inputs or in a device reduction */
  SBCI_ERR_NOT_CONVERGED = 5, /* step cap reached; best energies written */
  SBCI_ERR_TIMEOUT = 6,       /* a bounded device wait ran out */
  SBCI_ERR_CANCELLED = 7      /* request cancelled (serving) */
} sbci_status;

/* Arithmetic of the two-electron contraction inside sigma. */
typedef enum {
  SBCI_FP64 = 0,   /* FP64 gather, FP64 contraction, FP64 scatter.  For
                      npair <= 55 the contraction runs on the tensor cores by
                      exact BF16 integer slices of 56-bit scaled inputs (error-
                      free splitting, Ozaki, Ogita & Oishi 2012; FP64 accuracy);
                      else FP64 FMAs.  The environment variable
                      SBCI_FP64_CONTRACTION=dfma, read when a context is
                      created, selects the FMAs for every size.  With
                      density-fitted integrals ((ij|kl) of rank r by a pivoted
                      Cholesky, 2 (r + 2) < 0.9 npair) and npair > 55, the
                      FP64 FMA contraction uses the factored form
                      W = F M F^T, F = [L | kappa | delta], 2 (r + 2) npair
                      instead of npair^2 multiply-adds; SBCI_LOWRANK=0, read
                      when a context is created, turns it off. */
  SBCI_TF32X3 = 1, /* 3-term TF32 split on the tensor cores, FP32 accumulation
                      (about 2^-21 relative per product), n <= 14, and n = 15
                      with density-fitted integrals: there the full form's
                      operands exceed shared memory and the factored form
                      G = (D F)(F M)^T runs as two chained tensor-core products
                      per tile (SBCI_TC_LOWRANK=1, read when a context is
                      created, takes that form wherever it fits, 0 never);
                      singlet-sector
                      steps of spaces with at most 256 strings per spin run the
                      column-fused kernel (gather, contraction and scatter of one
                      column of the alpha part per CTA, no scratch in global
                      memory; SBCI_FUSED=0, read when a context is created,
                      keeps the tile kernel and scatter).  Where the tile
                      kernel's operands take more than half of shared memory
                      (npair > 55) it runs pipelined: epilogue warps drain one
                      TMEM accumulator while the next tile is contracted
                      (SBCI_TC_PIPE=0, read when a context is created, keeps
                      the plain kernel; the same results) */
  SBCI_BF16X3 = 2, /* 3-term BF16 split on the tensor cores (D_hi W_hi + D_hi W_lo +
                      D_lo W_hi, FP32 accumulation; about 2^-17 relative per
                      product), every orbital count up to 16: the tensor-core
                      mode of n = 15-16, where TF32 operands exceed shared memory */
  SBCI_FP32 = 3    /* FP32 SIMT contraction (reference for the split modes) */
} sbci_precision;

/* Solver parameters.  Defaults (sbci_params_init) are the paper's values for
 * calculations without frozen core (Section S1.3, S1.5). */
typedef struct {
  double eps0;      /* |E_{t+1}-E_t| < eps0 ... (Eq. S61), default 1e-10 */
  double r0;        /* ... and |z'| < r0, default 1e-5 */
  double b_th;      /* restart S62a: alpha>0, |b|<b_th, dE<eps1; 1e-2 */
  double eps1;      /* 1e-7 */
  double x_th1;     /* restart S62b: |k| < x_th1 or |k| > x_th2; 0.1 */
  double x_th2;     /* 1.2 */
  double r1;        /* restart S62c: |z'| > r1 and t > 0; 1.0 */
  int max_cycle;    /* restart when t+1 reaches max_cycle (S1.5); 20 */
  int max_sigma;    /* cap on H-products per state; 1000 */
  double guard;     /* |D_I - E0| floor of the preconditioner; 1e-8 */
  double gs_tol;    /* Gram-Schmidt drop tolerance (S1.1); 1e-14 */
  int sector;       /* 0: every determinant; 1: c = c^T (needs nalpha == nbeta) */
  int n_init;       /* determinants of the initial guess; 0 -> max(k, 2) */
  int init;         /* 0: lowest diagonal (S1.1); 1: caller vector c0 */
  int prec;         /* sbci_precision of the main stage; SBCI_FP64.  With a
                       low precision, each state runs SB steps with that sigma
                       until dE < mixed_eps and |z'| < mixed_r, then replaces
                       X by an FP64 H x and continues in FP64 to Eq. S61. */
  double mixed_eps; /* end of the low-precision stage: dE < mixed_eps ... ; 1e-8 */
  double mixed_r;   /* ... and |z'| < mixed_r; 1e-4 */
  int refine_max_sigma; /* H-products of the low-precision refinement stage per
                           state; X is made exact (one FP64 sigma) after every
                           max_cycle refinement steps, and when the budget is
                           spent, or two such windows end without Eq. S61 (the
                           low-precision sigma sits at its noise floor), the
                           state continues with FP64 sigma up to max_sigma;
                           300 */
  double start_noise; /* eta >= 0: every state's start becomes x0/|x0| + eta r/|r| with
                         r a seeded SplitMix64 vector in [-1,1) (X by one FP64 sigma of
                         r) and E_0 its Rayleigh quotient, before the projection of Eqs.
                         S4-S7.  SBCI1 keeps the spatial symmetry of its start; a small
                         full-symmetry part lets it reach the lowest remaining state in
                         symmetric molecules.  0 = the paper's starts.  0 */
  long long noise_seed; /* seed of r: element I of state alpha's vector is the SplitMix64
                           output of seed + 0x9E3779B97F4A7C15*(alpha*2^40 + I + 1),
                           top 53 bits mapped to [-1, 1).  0 */
  int init_stage;   /* 1: the H-products of the lowest-diagonal start (S1.1: H of each
                       start vector, giving the subspace matrix, E_0 and X_0) in the
                       stage precision prec instead of FP64, so that a mixed solve's
                       first FP64 H-product is its first re-sync (which replaces X by
                       an FP64 H x); no effect with prec = SBCI_FP64 or init = 1.
                       0 or 1, else SBCI_ERR_INVALID.  0 */
} sbci_params;

typedef struct {
  double energy;      /* total energy (electronic + e_core) */
  double residual;    /* |H x - E x| / |x| from the carried H-image */
  int converged;      /* 1 if Eq. S61 held (in FP64 after refinement) */
  int n_sigma;        /* H-products spent on this state (all precisions) */
  int n_sigma_fp64;   /* of which FP64 */
  int n_step;         /* SB steps */
  int n_restart[4];   /* restarts by cause: S62a, S62b, S62c, max_cycle */
  long long ctl_cycles; /* SM clock cycles the device controller (convergence and
                           restart tests, subspace solve) spent on this state */
  double s136_ratio;  /* energy-conservation health of the state (Section S4,
                         Eq. S136): geometric mean of |Delta E / ((2/c) Delta T)|
                         over its later steps with |Delta E| > 1e-6 hartree
                         (Delta E = E_t - E_{t+1}, the trace's s136 as the
                         denominator); near 1 when the classical energy of
                         Eq. 1 is conserved across updates; 0 if no step
                         qualified */
  int s136_steps;     /* steps in s136_ratio */
} sbci_report;

typedef struct {
  int state;          /* alpha */
  int t;              /* step index within the current restart cycle */
  double energy;      /* E_{t+1}, electronic (no e_core) */
  double b, c, k;     /* parameters of the step (Eqs. S23-S24, S53-S55) */
  double dE, dz;      /* |E_{t+1}-E_t| and |z'_{t+1}| */
  int event;          /* 0 none, 1 converged, 2..5 restart S62a/b/c/max_cycle,
                         6 low-precision stage ended: switch to FP64 refinement,
                         7 refinement budget, or two of its re-sync windows,
                           spent: the state continues with FP64 sigma from an
                           exact X (host record),
                         8 later-step coefficients undefined (zero denominator
                           in Eqs. S53-S55): the step was taken on the
                           first-step path from x */
  int prec;           /* sbci_precision of the sigma used in the step */
  double s136;        /* right-hand side of Eq. S136 for the update of this step,
                         (2/c_{t-1}) Delta T = (b_{t-1}/c_{t-1}) (y_{t+1}^T M y_{t+1}
                         - y_t^T M y_t) with the mass M = D - E_{t+1} (Section S4,
                         Eqs. S134-S136, indices of the update y_t -> y_{t+1});
                         its sign is that of c, which the sign of the subspace
                         eigenvector decides; NaN on first steps; 0 in host
                         records */
} sbci_trace_record;

/* Fills *p with the defaults listed above.  Returns SBCI_ERR_INVALID on NULL. */
sbci_status sbci_params_init(sbci_params *p);

/* Creates a context on the current CUDA device for one active space: the
 * Hamiltonian H whose lowest eigenpairs SBCI seeks (Eq. 1; the determinant
 * representation is the host program's, not specified by the paper).
 * Builds the string tables (host), the packed two-electron operator W
 * (one-electron part absorbed), the diagonal of H, and uploads them.
 * h1: host [norb*norb]; eri: host [norb^4] (ij|kl); both FP64, read only.
 * cuda_stream: a cudaStream_t to run on, or NULL for a library-owned stream.
 * On success *out owns all device memory until sbci_destroy.  Errors:
 * SBCI_ERR_INVALID for sizes outside the limits, h1 not symmetric or eri
 * without the 8-fold symmetry of real orbitals (1e-10 of the largest entry),
 * SBCI_ERR_NUMERIC for NaN/Inf inputs (both before any CUDA call),
 * SBCI_ERR_NOMEM / SBCI_ERR_CUDA from the device set-up (nothing leaks). */
sbci_status sbci_init_integrals(sbci_ctx **out, int norb, int nalpha, int nbeta,
                                const double *h1, const double *eri, double e_core,
                                void *cuda_stream);

/* n contexts of the same integrals, each as sbci_init_integrals would make it,
 * created in parallel on the library's host worker threads (no counterpart in
 * the paper: runtime support for batched and served solves, which make many
 * contexts at once).  out[n] receives them; cuda_streams: n streams (an entry
 * may be NULL: that context makes its own), or NULL for all.  The contexts
 * live on the calling thread's current device.  On an error none is left:
 * the ones made are destroyed, out[] is NULL and the first failing context's
 * status and message are returned. */
sbci_status sbci_init_integrals_many(sbci_ctx **out, int n, int norb, int nalpha, int nbeta,
                                     const double *h1, const double *eri, double e_core,
                                     void *const *cuda_streams);

/* Sizes of the determinant space: Ndet = Na*Nb; nlink = m(n-m+1) per string;
 * npair = n(n+1)/2.  Any output pointer may be NULL. */
sbci_status sbci_dims(const sbci_ctx *ctx, long long *ndet, int *na, int *nb,
                      int *nlink_a, int *nlink_b, int *npair);

/* Copies the device excitation table of one spin (0 alpha, 1 beta) to host
 * out[nstr*nlink*3] as (pair index, target string J, sign) triples in the
 * stored order: for each string I, for each occupied l ascending, for each
 * k in unocc(I) U {l} ascending, a+_k a_l |I> = sign |J>, pair = max(k,l)*
 * (max(k,l)+1)/2 + min(k,l). */
sbci_status sbci_string_table(const sbci_ctx *ctx, int spin, int *out);

/* D_I = <I|H|I> (electronic): the diagonal of the preconditioner
 * (D - E^0)^-1 (Eqs. 6-7, S31).  out: [Ndet] host (on_device = 0) or device. */
sbci_status sbci_diagonal(sbci_ctx *ctx, double *out, int on_device);

/* sigma = H c for nvec vectors, each [Ndet] (electronic H, no e_core): the
 * H-product of every SB step (Eqs. S9, S32).
 * c and sigma: host (on_device = 0) or device (on_device = 1) pointers to
 * nvec*Ndet doubles; they must not overlap.  prec: sbci_precision.
 * nvec = 0 does nothing.  Errors: SBCI_ERR_INVALID for NULL pointers,
 * nvec < 0 or a precision the context cannot run; SBCI_ERR_NUMERIC for
 * NaN/Inf in host input (device inputs are not scanned: non-finite values
 * propagate to sigma); SBCI_ERR_TIMEOUT when a bounded device wait of the
 * tensor-core kernels ran out (the context stays usable). */
sbci_status sbci_sigma(sbci_ctx *ctx, const double *c, double *sigma, int nvec,
                       int prec, int on_device);

/* Size of the fixed device scratch used by sbci_sigma_noalloc: 32 MiB,
 * enough for npair * Ndet <= 4,194,304 doubles (for example the 10-orbital,
 * 5+5-electron space: 55 * 63,504). */
#define SBCI_NOALLOC_SCRATCH_BYTES (32u * 1024u * 1024u)

/* sigma = H c in FP64 for one device vector, without allocating anything.
 * The paper has no counterpart: this is a library convenience for callers
 * that cannot call cudaMalloc at the time they need sigma -- code running
 * inside a stream capture, code in a framework that owns all device memory
 * through its own pool, or a latency-critical loop that cannot afford the
 * synchronisation an allocation implies.
 * c, sigma: device pointers to Ndet doubles each (caller-owned, not
 * overlapping).  cuda_stream: stream to run on, NULL for the context stream.
 * The call is asynchronous: sigma is ready when the stream reaches it.
 * Scratch: a file-scope static device array of SBCI_NOALLOC_SCRATCH_BYTES on
 * every GPU that loads the library, kept until process exit.  Its device
 * address is looked up on the first call on each device (with lazy module
 * loading that look-up is also when the array's memory is committed), so make
 * that first call before any stream capture.  Every call on a device shares the one
 * array: calls that overlap on the GPU (other streams, other threads, other
 * contexts) race and give wrong results; serialise them.  The array keeps
 * the last call's contents; every call overwrites all of the part it reads.
 * The context's device must be the current CUDA device (the array's address
 * is per device).
 * Errors: SBCI_ERR_INVALID for NULL arguments, a space whose scratch
 * (npair * Ndet * 8 bytes) exceeds the array, or a current device other than
 * the context's; SBCI_ERR_CUDA on a launch error.  Never calls cudaMalloc,
 * cudaFree or an allocating library routine. */
sbci_status sbci_sigma_noalloc(const sbci_ctx *ctx, const double *c, double *sigma,
                               void *cuda_stream);

/* Starts an SBCI1 solve for the k lowest states (Fig. 1A, Algorithm 1).
 * params may be NULL (defaults).  c0: host [Ndet] when params->init == 1,
 * else ignored (may be NULL).  Allocates the per-solve vectors. */
sbci_status sbci_begin(sbci_ctx *ctx, int k, const sbci_params *params, const double *c0);

/* One SB step of the current state (preconditioned projected residual,
 * sigma, 2x2/3x3 subspace solve, update, convergence/restart test).
 * rec (may be NULL) receives the step record.  *done = 1 when all k states
 * have ended.  Returns SBCI_ERR_NOT_CONVERGED when a state hit max_sigma
 * (the solve then moves on to the next state). */
sbci_status sbci_step(sbci_ctx *ctx, sbci_trace_record *rec, int *done);

/* Results of the solve: energies [k] (total), vecs [k*Ndet] host (or NULL),
 * rep [k] (or NULL). */
sbci_status sbci_finish(sbci_ctx *ctx, double *energies, double *vecs, sbci_report *rep);

/* begin + steps until done + finish.  Returns SBCI_ERR_NOT_CONVERGED if any
 * state stopped at its cap (results still written). */
sbci_status sbci_solve(sbci_ctx *ctx, int k, const sbci_params *params, const double *c0,
                       double *energies, double *vecs, sbci_report *rep);

/* Solves n contexts (1 <= n <= 64) for their k lowest states together: the
 * solves with a TF32x3 sigma and n_orb <= 14 advance in one CUDA-graph loop of
 * batched persistent kernels over a device job table (see sbci_server_*);
 * others are solved one after the other.  params as in sbci_solve (init must
 * be 0).  energies: host [n][k] totals; rep: host [n][k] or NULL; launches
 * (nullable): kernels this call launched (per batched loop body: update,
 * projection, the sigma kernels its solves need -- tensor-core tile kernel and
 * scatter, or the column-fused kernel of singlet-sector solves with at most
 * 256 strings per spin -- the symmetric finish of sector solves, and the end
 * kernel; plus the host-driven ones).  Each context afterwards holds its
 * finished solve (sbci_finish, sbci_trace).  The per-solve host work between
 * batch rounds (initial guesses, FP64 re-syncs and verifications, the next
 * state's start) runs in parallel on the library's host worker threads, so
 * contexts with their own CUDA streams overlap it; SBCI_HOST_THREADS=0 (read
 * on first use) keeps it on the calling thread.  Results do not depend on it. */
sbci_status sbci_solve_batch(sbci_ctx **ctx, int n, int k, const sbci_params *params, double *energies,
                             sbci_report *rep, long long *launches);

/* SBCI2 (Algorithm 2, Sections S2.1-S2.5, Fig. 1B): the k lowest states,
 * found one by one from the lowest while the pair (alpha, alpha+1) is updated
 * together (two H-products per step, a 6x6 canonically orthogonalised
 * subspace, coefficients of Eqs. S93, S112, S116, S117, S121, restarts S130a-c
 * and max_cycle2); the highest state runs SBCI1.  FP64 sigma.  Readings where
 * the paper is silent: start vectors from max(k, n_init or 2) lowest-diagonal
 * vectors (S74-S76); a later pair's upper start is projected against the
 * stored states and the new lower vector, normalised, with X_0 = H x_0 by one
 * H-product and E_0 its Rayleigh quotient; the preconditioner shift is E_t of
 * state 0 in the ground pair, E_c^0 afterwards; x_{t+1} and X_{t+1} are taken
 * as k v and its H-image (the vectors Eqs. S124-S125 give in exact arithmetic);
 * undefined later-step coefficients take the first-step path; a restart keeps
 * x/|x|, X/|x| and takes the first-step path.
 * params: NULL for defaults; needs prec = SBCI_FP64, init = 0, start_noise = 0
 * (else SBCI_ERR_INVALID).  max_cycle2: restart period of the pairs, 0 -> 10
 * (Section S2.5); params->max_cycle applies to the last state.  Energies are
 * in the order the states were found (the pair's lower state first); rep as
 * sbci_solve (per state: H-products and steps while it was the lower state);
 * sbci_trace gives the step records of the pairs (b, c, k: b^{aa}, c^{aa},
 * k_0) followed by the last state's.  The pair steps are driven from the
 * host (the small eigen-problems on the host); SBCI_SBCI2_DEVICE=1, read when
 * a context is created, runs them on a device controller as a CUDA-graph
 * loop instead (the same steps; slower on GB300, whose FP64 rate makes the
 * one-thread 6x6 eigen-solves dearer than the host round trips). */
sbci_status sbci_solve_sbci2(sbci_ctx *ctx, int k, const sbci_params *params, int max_cycle2,
                             double *energies, double *vecs, sbci_report *rep);

/* Lowest k eigenpairs by block Davidson-Liu (Davidson 1975; Liu 1978) on the
 * same FP64 sigma: the method the paper compares SBCI with (Introduction;
 * Materials and Methods, where it runs with the preconditioner
 * (D - E^0 I)^-1).  It keeps the whole subspace V and H V (up to max_space
 * vectors each) where SBCI1 keeps x, y, z and their H-images.  Schedule:
 *   start: determinants by ascending (D_I, I), symmetrised when
 *     params->sector = 1, Gram-Schmidt orthonormalised (dropped below gs_tol),
 *     until max(k, n_init or 2) vectors;
 *   each iteration: Ritz pairs of (T + T^T)/2, T = V^T H V; residuals
 *     r_a = H x_a - theta_a x_a; state a has converged when
 *     |theta_a - theta_a(previous iteration)| < eps0 and |r_a| < r0 (Eq. S61);
 *   when m + (unconverged states) > max_space, V and H V collapse onto the
 *     k Ritz vectors;
 *   per unconverged state, in order: t = r_a / (D - theta_a) (|D_I - theta_a| <
 *     guard -> sign * guard), symmetrised in the sector, projected twice against
 *     V, dropped if |t|^2 < gs_tol |t_0|^2, normalised, appended (one sigma);
 *   an iteration that appends nothing ends the solve (converged if every
 *     |r_a| < r0); so does the cap of max_sigma * k H-products.
 * params: NULL for defaults; eps0, r0, guard, gs_tol, sector, n_init and
 *   max_sigma are used, the other fields ignored (sigma is always FP64).
 * max_space: subspace limit, 0 -> max(12, 4k); 2k <= max_space <= 64.
 * k: 1..8.  energies: host [k] totals.  vecs: host [k*Ndet] Ritz vectors or
 * NULL.  rep: host [k] or NULL -- residual |r_a|, converged, n_sigma (total
 * H-products of the solve), n_step (iterations), n_restart[0] (collapses).
 * vector_bytes (nullable): device bytes of the subspace buffers
 * (2 (max_space + k) Ndet doubles), allocated for the call and freed before
 * it returns.  Returns SBCI_ERR_NOT_CONVERGED when it stops short (results
 * written), SBCI_ERR_INVALID for bad arguments or fewer than k start vectors,
 * SBCI_ERR_NOMEM when the buffers do not fit. */
sbci_status sbci_davidson(sbci_ctx *ctx, int k, const sbci_params *params, int max_space,
                          double *energies, double *vecs, sbci_report *rep, long long *vector_bytes);

/* Copies up to cap trace records of the last solve; *n = records available.
 * The records are the per-step quantities the paper plots (Fig. 3: E_t, b,
 * c, k, |E_{t+1} - E_t|, |z'|) plus the events of the solve. */
sbci_status sbci_trace(const sbci_ctx *ctx, sbci_trace_record *buf, int cap, int *n);

/* Per-kernel statistics of the library's own launches on the context stream
 * (no counterpart in the paper). */
typedef struct {
  char name[32];       /* kernel family, e.g. "sigma_gather_contract" */
  long long launches;  /* launches since the last sbci_profile call */
  double total_ms;     /* summed CUDA-event time of those launches (0 if timing off) */
} sbci_kernel_stat;

/* Resets the statistics.  Launches are always counted (including the kernels
 * a solve's CUDA graph runs).  enable = 1 also brackets every launch with
 * CUDA events on the context stream; solves then launch their step kernels
 * one by one instead of through the graph, so that each can be timed. */
sbci_status sbci_profile(sbci_ctx *ctx, int enable);

/* Waits for the recorded events and copies up to cap entries; *n = families. */
sbci_status sbci_profile_read(sbci_ctx *ctx, sbci_kernel_stat *out, int cap, int *n);

/* Kernel timing of the batch engine that sbci_solve_batch uses on the current
 * device (no counterpart in the paper).  Resets its statistics; enable = 1
 * makes later sbci_solve_batch calls on this device launch the kernels of
 * every batched loop body one by one, each bracketed by CUDA events on the
 * engine's stream, instead of through the graph loop (same arithmetic). */
sbci_status sbci_batch_profile(int enable);

/* Waits for the recorded events and copies up to cap entries (families
 * "batch_update", "batch_project", "batch_gather_contract_tc",
 * "batch_fused_column", "batch_scatter", "batch_symfinish", "batch_end",
 * then "batch_host_halted": launches = halted solves handled on the host
 * between rounds, total_ms = the host wall time of that handling (their FP64
 * re-syncs, verifications and state changes, with the GPU work it waits
 * for)); *n = 8.  A family that a class does not launch stays at zero. */
sbci_status sbci_batch_profile_read(sbci_kernel_stat *out, int cap, int *n);

/* Launch shapes of the batch engine on the current device, one record per
 * class of job tables met so far (no counterpart in the paper): the operand
 * sizes of its tile-kernel and column-kernel jobs and the kernels its loop
 * body launches.  The autotuner fills ctas[] once it has timed every
 * candidate (tuned = 1). */
typedef struct {
  int Kp, Np;            /* tile-kernel operand class (padded pair counts) */
  int smem_bytes;        /* dynamic shared memory of a tile-kernel CTA */
  int tc_per_sm_max;     /* tile-kernel CTAs that fit one SM */
  int tuned;             /* 1 once the autotuner has chosen */
  int ctas[7];           /* update, projection, tensor-core tile, fused column, scatter,
                            symmetric finish, end */
  int fKp, fNp;          /* column-kernel operand class (the singlet-sector solves
                            with at most 256 strings per spin) */
  int fused_smem_bytes;  /* dynamic shared memory of a column-kernel CTA */
  int kernels;           /* bit k set: kernel k of ctas[] is launched in each loop body */
} sbci_batch_class;

/* Copies up to cap records; *n = classes. */
sbci_status sbci_batch_classes(sbci_batch_class *out, int cap, int *n);

/* ---------------------------------------------------------------------------
 * Serving: continuous batching of solves on one GPU (no counterpart in the
 * paper, which runs one solve at a time; this is the request loop around the
 * same SBCI1 solve).  Requests are admitted from a FIFO queue into slots while
 * a slot is free and the request's device-memory footprint fits the budget;
 * each admitted solve keeps its state resident and runs its SB steps as a
 * CUDA-graph loop on its own stream, so solves overlap on the device.  One
 * host thread drives the server; calls are not thread-safe. */
typedef struct sbci_server sbci_server;

/* mem_budget_bytes: device memory the server may hold for admitted solves;
 * max_slots: solves in flight at once (1..1024). */
sbci_status sbci_server_create(sbci_server **out, size_t mem_budget_bytes, int max_slots);

/* Queues one solve of the k lowest states (1 <= k <= 8).  h1, eri, e_core as
 * in sbci_init_integrals (copied at the call); params may be NULL.
 * *ticket identifies the request.  SBCI_ERR_NOMEM if its footprint alone
 * exceeds the budget. */
sbci_status sbci_server_submit(sbci_server *sv, int norb, int nalpha, int nbeta, const double *h1,
                               const double *eri, double e_core, int k, const sbci_params *params,
                               long long *ticket);

/* Non-blocking progress: admits what fits, handles every slot whose graph
 * round has finished (controller event, next round or retirement).  Outputs
 * (nullable): solves in slots, requests still queued. */
sbci_status sbci_server_progress(sbci_server *sv, int *n_active, int *n_queued);

/* *done = 1 once the request has finished; then energies [k] (total),
 * rep [k] and times [2] = {queueing seconds, latency seconds from submit to
 * completion} are written (each nullable) and the solve's status returned;
 * for an error status, sbci_last_error() then gives that solve's message. */
sbci_status sbci_server_poll(sbci_server *sv, long long ticket, int *done, double *energies,
                             sbci_report *rep, double *times);

/* on = 1 (the default): admitted solves with a TF32x3 sigma and n <= 14 are
 * advanced together by one CUDA-graph loop of batched persistent kernels that
 * walk a device job table (a work queue of (solve, block) items); on = 0: every
 * solve runs its own graph loop on its own stream.  Only while no solve is
 * admitted. */
sbci_status sbci_server_set_batching(sbci_server *sv, int on);

/* Waits for in-flight rounds and frees every slot.  NULL is a no-op. */
void sbci_server_destroy(sbci_server *sv);

/* Thread-local message of the last error in this thread ("" if none). */
const char *sbci_last_error(void);

/* Frees everything the context owns (after waiting for its stream).  NULL
 * is a no-op.  Device and pinned host buffers up to 256 MiB go to the
 * library's buffer cache rather than back to CUDA (see sbci_pool_trim). */
void sbci_destroy(sbci_ctx *ctx);

/* The library's buffer cache (no counterpart in the paper: runtime support).
 * Contexts and solves allocate their device and pinned host buffers through
 * it; a freed buffer of at most 256 MiB is kept (up to 2 GiB cached in all,
 * per device for device memory) and serves the next request of the same
 * rounded size, so creating and destroying contexts in a loop does not call
 * cudaMalloc / cudaFree (which synchronises the device) each time.
 * sbci_pool_stats: bytes cached now and the requests served from the cache
 * (hits) and from CUDA (misses) since the process started (each pointer may
 * be NULL).  sbci_pool_trim: returns every cached buffer to CUDA; SBCI_ERR_CUDA
 * if a free failed.  Thread-safe. */
sbci_status sbci_pool_stats(size_t *cached_bytes, long long *hits, long long *misses);
sbci_status sbci_pool_trim(void);

#ifdef __cplusplus
}
#endif

#endif /* SBCI_H */
