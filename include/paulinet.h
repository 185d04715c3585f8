/*
 * paulinet.h -- C ABI of libpaulinet.so, the GB300 (sm_103a) hot path of
 * PauliNet variational quantum Monte Carlo (Hermann, Schaetzle & Noe,
 * arXiv:1909.08423).
 *
 * Conventions shared by every call
 *  - Return value: PN_OK (0) or a PN_E* code; pn_last_error() gives a
 *    thread-local message for the last failure on the calling thread.
 *  - Units: bohr and hartree.  Walker positions r are walker-major
 *    [W][N][3] float64 with the n_up up-spin electrons first.
 *  - Buffers may be device pointers or host pointers (pageable or pinned);
 *    the library asks the CUDA runtime which.  Device buffers are used in
 *    place and the call is asynchronous on `stream` (a cudaStream_t, NULL for
 *    the legacy default stream).  If any buffer of a call is a host pointer,
 *    the library stages it through its own device buffers on `stream` and
 *    synchronises `stream` before returning.
 *  - Ownership: the caller owns every buffer it passes; the library copies
 *    what it keeps (pn_init_system, pn_set_params) and owns its handles.
 *  - A system handle is not safe to use from two host threads at once and
 *    its direct calls share one workspace: do not overlap two calls on one
 *    handle on different streams.  The serving loop (pn_server_*) owns
 *    separate workspaces per slot.
 */
#ifndef PAULINET_H
#define PAULINET_H

#include <stddef.h>
#include <stdint.h>

#ifdef __cplusplus
extern "C" {
#endif

enum {
  PN_OK = 0,
  PN_EINVAL = 1,      /* bad argument, size beyond a compiled limit        */
  PN_ENOMEM = 2,      /* device allocation failed                          */
  PN_EBUDGET = 3,     /* job can never fit the server's memory budget      */
  PN_ENOTREADY = 4,   /* job still queued or running                       */
  PN_ETIMEOUT = 5,    /* a bounded wait ran out                            */
  PN_EDEVICE = 6,     /* CUDA runtime error                                */
  PN_ECANCELLED = 7   /* job was cancelled                                 */
};

enum { PN_FP64 = 0, PN_MIXED = 1 };

/* Per-walker status word written by the evaluation calls. */
enum { PN_WALKER_OK = 0, PN_WALKER_NONFINITE = 1, PN_WALKER_SINGULAR = 2 };

/* Compiled limits (checked by pn_init_system). */
#define PN_MAX_ELECTRONS 32
#define PN_MAX_SPIN 16
#define PN_MAX_ORBITALS 32
#define PN_MAX_DETS 64
#define PN_MAX_NUCLEI 16
#define PN_MAX_LAYERS 8
#define PN_MAX_DIM 256

typedef struct pn_system_s* pn_system_t;

/*
 * System description (all host pointers; copied by pn_init_system).
 *
 * Eq. (ansatz) of the paper:
 *   psi(r) = exp(gamma + J) sum_p c_p det[phi~_up] det[phi~_dn],
 *   phi~_{mu i} = phi_mu(r_i) f_{mu i}(r),  f = 1 + kappa(x_i^(L)),
 *   J = eta(sum_i x_i^(L)), gamma = sum_{i<j} -c_ij/(1 + r_ij) with
 *   c_ij = 1/4 (same spin) or 1/2 (opposite spin) (Methods, cusp conditions).
 *
 * Basis (Methods, computational details; the paper uses 6-311G):
 *   shell s is centred on nucleus shell_center[s] with l = shell_l[s]:
 *   l = 0, 1, 2: Cartesian Gaussians x^a y^b z^c sum_k d_k exp(-alpha_k r^2)
 *   with components (1) | (x,y,z) | (xx,xy,xz,yy,yz,zz); l = -1: Slater 1s
 *   d exp(-zeta r) (one "primitive" holds zeta and d).  Primitives of shell s
 *   are consecutive in prim_exp/prim_coef; coefficients are used as given.
 *   mo_coeffs is [n_b][n_orb] (basis-function-major): phi = C^T chi.
 * Determinants: occ_up [n_det][n_up], occ_dn [n_det][n_dn] orbital indices,
 *   ci [n_det] the expansion coefficients c_p.
 * Network (Methods, PauliNet extension of SchNet; Table 2): D = dim x,
 *   Zd = dim z, K = number of distance features, L = interaction layers,
 *   r_c the feature cutoff.  params is the flat float64 vector
 *   (n_params = pn_num_params_for(D, Zd, K, L, M, n_orb)) in this order,
 *   every linear map stored [in][out] (y = x W + b), Hw = max(K, Zd):
 *     x0[D], Y[M][Zd],
 *     for n < L:  hW[D][Zd], hb[Zd],
 *                 for c in (same, anti, nuc): W1[K][Hw], b1[Hw], W2[Hw][Zd], b2[Zd]
 *                 for c in (same, anti, nuc): GW[Zd][D], Gb[D]
 *     eta:   W1[D][D] b1[D] W2[D][D] b2[D] W3[D][1] b3[1]
 *     kappa: W1[D][D] b1[D] W2[D][D] b2[D] W3[D][n_orb] b3[n_orb]
 *   Activation between layers: shifted softplus ln(e^x/2 + 1/2).
 * Nuclear cusps (Methods, cusp conditions; Ma et al. 2005): with use_cusp,
 *   inside r_c = 0.5/Z_I of each nucleus the l=0 Gaussian part of every
 *   orbital is replaced by C + s exp(quartic(r)) matching value, slope and
 *   curvature at r_c and Kato's cusp at the nucleus.  cusp_phi0 [n_orb][M]
 *   gives the s part's value at the nucleus (NULL: keep the Gaussian value).
 * precision: PN_FP64 (every step in float64) or PN_MIXED (network in
 *   float32, orbitals, determinants, log-sum, Laplacian sum and Coulomb
 *   terms in float64).
 * max_walkers: walkers per chunk of the library's workspace (the workspace
 *   grows with it; calls with more walkers run chunk by chunk).
 */
typedef struct pn_system_desc {
  int M;
  const double* Z;           /* [M]   */
  const double* R;           /* [M][3] */
  int n_shells;
  const int* shell_center;   /* [n_shells] */
  const int* shell_l;        /* [n_shells] */
  const int* shell_nprim;    /* [n_shells] */
  const double* prim_exp;    /* [sum nprim] */
  const double* prim_coef;   /* [sum nprim] */
  int n_up, n_dn, n_orb;
  const double* mo_coeffs;   /* [n_b][n_orb] */
  int n_det;
  const int* occ_up;         /* [n_det][n_up] */
  const int* occ_dn;         /* [n_det][n_dn] */
  const double* ci;          /* [n_det] */
  int D, Zd, K, L;
  double r_c;
  const double* params;      /* [n_params] */
  int64_t n_params;
  const double* cusp_phi0;   /* [n_orb][M] or NULL */
  int use_cusp, use_gamma;
  int precision;             /* PN_FP64 | PN_MIXED */
  int max_walkers;           /* workspace chunk (walkers) */
  /* Ablation variants of the ansatz (Results, the comparison of single and
   * multiple determinants with and without backflow): no_jastrow = 1 removes
   * the Jastrow factor (J = 0), no_backflow = 1 the backflow (f = 1).  The
   * removed head's parameters stay in the layout; its last map is held at
   * zero on the device and its gradient entries are returned as zero. */
  int no_jastrow, no_backflow;
} pn_system_desc;

/* Number of network parameters for the given sizes (layout above). */
int64_t pn_num_params_for(int D, int Zd, int K, int L, int M, int n_orb);

/* Validate, precompute the cusp coefficients (host, float64), upload the
 * system and allocate the workspace for max_walkers walkers.
 * Errors: PN_EINVAL (sizes, indices, limits), PN_ENOMEM, PN_EDEVICE. */
int pn_init_system(const pn_system_desc* desc, pn_system_t* out);
int pn_destroy_system(pn_system_t sys);

/* Replace the network parameters (same layout; host or device pointer).
 * Synchronous. */
int pn_set_params(pn_system_t sys, const double* params, int64_t n_params);
int64_t pn_num_params(pn_system_t sys);
/* Bytes of device workspace held by the handle. */
size_t pn_workspace_bytes(pn_system_t sys);

/* ln|psi| and sign(psi) of Eq. (ansatz) for W walkers.
 * r [W][N][3]; logabs, sign [W] float64; status [W] int (PN_WALKER_*). */
int pn_eval_logpsi(pn_system_t sys, const double* r, int W, double* logabs,
                   double* sign, int* status, void* stream);

/* Local energy E_loc = -1/2 lap psi / psi + V (Eq. monte-carlo) with the
 * Laplacian carried forward through the whole ansatz as a jet (value, 3N
 * first derivatives, Laplacian).  eloc, logabs, sign [W] float64 (logabs and
 * sign may be NULL); status [W] int or NULL. */
int pn_eval_local_energy(pn_system_t sys, const double* r, int W, double* eloc,
                         double* logabs, double* sign, int* status,
                         void* stream);

/* Intermediate quantities of the value pass, for step-by-step checks:
 * phi [W][N][n_orb] orbitals, J [W], f [W][N][n_orb] backflow,
 * ld [W][n_det] ln|det_up det_dn| per determinant (each may be NULL). */
int pn_eval_components(pn_system_t sys, const double* r, int W, double* phi,
                       double* J, double* f, double* ld, void* stream);

/* ln|psi| and sign(psi) like pn_eval_logpsi, for callers that cannot
 * allocate device memory while they evaluate (a latency-bound loop that must
 * not wait on the allocator, a process that reserves its memory once at
 * start-up).  The paper has no counterpart:
 * this is a deployment variant of the value pass.  The call allocates
 * nothing: its intermediates live in one fixed 16 MiB file-scope device
 * array that every GPU loading the library holds until the process exits.
 * All buffers must be device pointers, and the handle's device must be
 * current.  W is limited by that array (it holds only the value pass's
 * intermediates: about 700 walkers of a four-electron, D = 64 system in
 * PN_FP64); a larger W returns PN_EINVAL
 * with the limit in pn_last_error() and launches nothing.  The first call on
 * each device looks up the array's device address (cudaGetSymbolAddress);
 * make that first call before any stream capture.  Every call shares the one
 * array, so calls that overlap on the GPU (other streams, other threads)
 * race: serialise them.  No part of the array has to start at zero. */
int pn_eval_logpsi_static(pn_system_t sys, const double* r, int W,
                          double* logabs, double* sign, int* status,
                          void* stream);

/* n_steps Metropolis steps for each walker (Methods, ansatz optimisation:
 * sampling of |psi|^2; Gaussian all-electron proposal of width sigma):
 * r' = r + sigma xi, accept iff u < exp(2 (ln|psi(r')| - ln|psi(r)|)).
 * r [W][N][3] and logabs [W] are updated in place (logabs must hold
 * ln|psi(r)| on entry).  xi and u come from Philox4x32-10 with key = seed
 * and counter (j, walker0 + w, step, step >> 32) for step = step0 .. step0 +
 * n_steps - 1 (walker0 = 0 here).  n_accept (one int64, may be NULL) receives
 * the number of accepted moves summed over walkers and steps. */
int pn_metropolis_step(pn_system_t sys, double* r, double* logabs, int W,
                       int n_steps, double sigma, uint64_t seed, uint64_t step0,
                       int64_t* n_accept, void* stream);

/* ln|psi| and its gradient with respect to the electron positions,
 * drift [W][N][3] = grad_r ln|psi| (the quantity the Langevin proposal
 * follows; Methods, ansatz optimisation, sampling).  By default it is formed
 * in reverse mode (one value pass kept on the handle's tape, then the chain
 * back from ln|psi| to the pair distances and orbitals; the tape is
 * allocated on first use and kept); PN_OPT_DRIFT = 0 selects the jet pass
 * of pn_eval_local_energy instead.  logabs may be NULL.  Host or device
 * buffers; a call with a host buffer returns after the results are
 * written. */
int pn_eval_drift(pn_system_t sys, const double* r, int W, double* logabs,
                  double* drift, void* stream);

/* E_loc, ln|psi| and sign along a line through configuration space
 * (Results, the one-dimensional scan of the wave function and its local
 * energy in LiH): point k of npts is the configuration r0 [N][3] with
 * electron `electron` at r0[electron] + t_k dir, t_k = t0 + k (t1 - t0) /
 * (npts - 1).  Passing the line through a nucleus or another electron shows
 * the cusps: with the cusp splice and gamma, E_loc stays finite at the
 * coalescence points.  r0 is host or device; dir is a HOST array of three
 * doubles; eloc [npts] (required), logabs, sign [npts] and status [npts]
 * (may be NULL) are host or device.  Uses the handle's workspace in chunks;
 * allocates nothing. */
int pn_eval_line_scan(pn_system_t sys, const double* r0, int electron,
                      const double* dir, double t0, double t1, int npts,
                      double* eloc, double* logabs, double* sign, int* status,
                      void* stream);

/* n_steps Langevin (drift-diffusion) Metropolis-Hastings steps for each
 * walker (Methods, ansatz optimisation: Langevin Monte Carlo after Umrigar
 * et al., its radial proposal replaced by clipping the step length at the
 * nearest nucleus).  All electrons move at once:
 *   r' = r + c(r) + sqrt(tau) xi,  c_e = tau drift_e, shortened to the
 *        distance from r_e to its nearest nucleus when it is longer,
 *   accept iff u < |psi(r')/psi(r)|^2 T(r' -> r) / T(r -> r'),
 *   T(x -> y) = exp(-|y - x - c(x)|^2 / (2 tau)).
 * xi and u come from the same Philox4x32-10 stream layout as
 * pn_metropolis_step.  r [W][N][3], logabs [W] and drift [W][N][3] must be
 * DEVICE buffers holding ln|psi(r)| and grad ln|psi(r)| on entry
 * (pn_eval_drift); they are updated in place.  The drift at each proposal
 * is formed as in pn_eval_drift (PN_OPT_DRIFT).  n_accept (one int64, host
 * or device, may be NULL) receives the accepted moves over walkers and
 * steps.  tau > 0 is the time step; the paper tunes it for 57 % acceptance,
 * which is left to the caller.  PN_EINVAL for host buffers or tau <= 0. */
int pn_langevin_step(pn_system_t sys, double* r, double* logabs, double* drift,
                     int W, int n_steps, double tau, uint64_t seed,
                     uint64_t step0, int64_t* n_accept, void* stream);

/* Implementation options of a handle (they change speed, not results
 * beyond floating-point rounding).
 * PN_OPT_FUSED_SAMPLER (default 4 for PN_MIXED, 1 for PN_FP64): run
 *   Metropolis steps in one launch that
 *   keeps walkers in shared memory for all steps -- one warp per walker for
 *   small systems (up to 24 KiB of state per walker; weights read through
 *   L1/L2), else a tile of walkers per block; 2 forces the tile kernel; 3
 *   the warp kernel with its block's warps walking the layers in lockstep
 *   and each weight block bulk-copied (TMA) into shared memory one stage
 *   ahead; 4 (PN_MIXED) the tensor-core sampler -- a block per tile of
 *   walkers whose electrons and pairs fill 128-row tcgen05 tiles, every
 *   linear map one MMA group with three-piece bf16 operands and weights
 *   bulk-copied (TMA) one stage ahead -- falling back, where the tiles do
 *   not fit, to 1 for embeddings up to 64 wide and to 0 beyond (there the
 *   staged value pass is the faster); 0 (or a system too large for one
 *   tile) uses one kernel per stage.
 * PN_OPT_TENSOR_CORES (PN_MIXED only; default 7): a mask of the float32
 *   linear layers that run on tcgen05 (maps of at least 8192 rows whose
 *   weight fits in shared memory; the rest on CUDA cores): 1 = interaction
 *   layers of the local-energy jet, 2 = its heads, 4 = value passes (ln|psi|
 *   and the gradient's recomputation).  Each float32 operand is split into
 *   three bf16 pieces and the six piece products of weight down to 2^-16
 *   accumulate in tensor memory, the leading products in an accumulator of
 *   their own: measured against float64, at most 1.6e-7 of sum |x w| per
 *   element for the network's maps (CUDA-core float32: 3.0e-7).  The Python
 *   helper paper_1909_08423_gb300.precision.calibrate measures the E_loc
 *   error of each mask against PN_FP64 on a system's sampled walkers.
 * PN_OPT_DRIFT (default 1): how pn_eval_drift and pn_langevin_step form
 *   grad_r ln|psi| -- 1 reverse mode (work linear in the electron count),
 *   0 the forward jet pass (3N + 2 rows per electron).
 * PN_OPT_GUARD (PN_MIXED only; default 50): the local-energy guard of
 *   pn_eval_local_energy, value = tau in micro-hartree, 0 = off.  The
 *   float32 network's rounding reaches E_loc through the determinants and
 *   the squared gradient, and a few walkers in ten thousand amplify it past
 *   1e-4 Ha, with no cheap per-walker predictor of which.  With the guard on,
 *   every workspace chunk is evaluated a second time from the same network
 *   output with different rounding (see PN_OPT_GUARD_PROBE) and every walker
 *   whose two energies differ by more than tau, or not finitely, is
 *   evaluated again in float64 -- its linear maps and filter nets as
 *   float32 pairs (about 44 bits; float32 issue rates are 64 times the
 *   float64 rate on this part), everything else in float64 -- and returned
 *   with those E_loc, ln|psi|, sign and status.  Each guarded chunk reads
 *   one count back to the host (the call then synchronises its stream once
 *   per chunk).  With positions and outputs in device memory the flagged
 *   walkers of successive chunks are re-evaluated together (up to 1024 at a
 *   time); with host buffers, each chunk's before its outputs are copied
 *   (the same values either way).  pn_guard_count reports how many walkers
 *   were re-evaluated.
 * PN_OPT_GUARD_PROBE (default 2): the guard's second evaluation.  2: the
 *   first pass's backflow and Jastrow jets perturbed by +-2^-19 relative
 *   plus a third of 2^-19 at the scale of the heads' terms (sum_k |x_k|
 *   |W_kn| of the last map of each head: rounding enters an output at that
 *   scale, which cancellation can make far larger than the output), with a
 *   deterministic sign per element, then the determinants and E_loc formed
 *   again.  Measured at the default tau on 16384-walker samples from
 *   |psi|^2 (6 per system): 1.8-2.2 % (H10 chain) and 2.3-2.8 % (N2 shape)
 *   of walkers re-evaluated, every remaining error at most 9.0e-5 Ha.
 *   1: the relative perturbation alone: 1.0-1.3 % and 0.46-0.66 %
 *   re-evaluated, the remaining errors at most 1.1e-4 Ha on those samples
 *   (one walker of the 196608 above 1e-4 Ha).  0: the heads (the Jastrow and
 *   backflow maps) evaluated again on the other unit (tensor cores if they
 *   ran on CUDA cores, and back), then the determinants and E_loc.
 * PN_OPT_DET_TABLE (default 1): how the forward passes form the
 *   determinants (and, in the local-energy pass, their gradients and
 *   Laplacians) -- 1 by the table method where the system allows it (every
 *   determinant reached from determinant 0 by at most 4 orbital
 *   replacements per spin, at most 8 electrons and 8 virtual orbitals per
 *   spin): det A_p = s_p det A_0 det(T[holes, particles]) with T = A_0^-1 A,
 *   so that the 3N tangents and the Laplacian of all determinants follow
 *   from those of determinant 0 and of T; a walker whose determinant-0
 *   block has a 1-norm condition number beyond 1e3 (jet) or 1e5 (value
 *   pass) is computed block by block; 0 block by block for every walker; 2
 *   the table kernel with every walker on its block-by-block path (a test of
 *   that path). */
enum { PN_OPT_FUSED_SAMPLER = 1, PN_OPT_TENSOR_CORES = 2, PN_OPT_DRIFT = 3, PN_OPT_GUARD = 4, PN_OPT_DET_TABLE = 5,
       PN_OPT_GUARD_PROBE = 6 };
int pn_set_option(pn_system_t sys, int option, int value);

/* Walkers the local-energy guard (PN_OPT_GUARD) re-evaluated in float64
 * since the last call, summed over calls; resets the count.  Synchronises
 * the device.  0 for PN_FP64 handles. */
int pn_guard_count(pn_system_t sys, int64_t* n);

/* Synchronises the device and reports whether any of the handle's kernels
 * gave up a bounded wait since the last check (PN_ETIMEOUT; the affected
 * outputs are invalid) -- PN_OK otherwise. */
int pn_device_status(pn_system_t sys);

/* Initial walkers: electron e at R[nucleus(e)] + N(0, 1) per coordinate
 * (Methods: Gaussians around the nuclei), nucleus(e) from the list of nuclei
 * repeated Z_I times, up electron k -> entry 2k, down electron k -> 2k+1
 * (modulo the list length); normals from the Philox stream at step 2^64-1. */
int pn_init_walkers(pn_system_t sys, double* r, int W, uint64_t seed, void* stream);

/* grad[P] = sum_w cotangent[w] d ln|psi(r_w)| / d theta over the network
 * parameters (layout above) -- the backward pass needed by Eq. (trainig).
 * The value pass is recomputed chunk by chunk so that the stored activations
 * stay within mem_budget_bytes (0: room for max(max_walkers, 256) walkers).
 * A budget below one walker's tape returns PN_EINVAL. */
int pn_grad_logpsi(pn_system_t sys, const double* r, int W, const double* cotangent,
                   double* grad, size_t mem_budget_bytes, void* stream);

/* Smooth clipping of local energies (Methods, ansatz optimisation): with
 * m = median, d = mean |E - m|, Lq = q d: E' = E inside |E - m| <= Lq, else
 * m + sgn(E - m) Lq (1 + ln(|E - m| / Lq)).  Also writes, if non-NULL,
 * cot[W] = 2 (E'_w - mean E') / W, the per-walker weights of the loss
 * gradient in Eq. (trainig).  W <= 2^26: up to 16384 walkers one block
 * sorts the energies in shared memory; beyond, a bitonic network sorts
 * them in global memory (stream-ordered scratch of 8 bytes per walker,
 * rounded up to a power of two). */
int pn_clip_local_energy(const double* eloc, int W, double q, double* out,
                         double* cot, void* stream);

/* ---------------------------------------------------------------------
 * Serving loop: a persistent host thread that admits jobs by device-memory
 * footprint as slots free up and runs admitted jobs concurrently on
 * separate streams, one host thread per slot (continuous batching across
 * molecules).  Mixed jobs' local energies carry the guard of PN_OPT_GUARD
 * with the system handle's tau (their footprint includes its float64
 * workspace).
 */
typedef struct pn_server_s* pn_server_t;

/* One AdamW step for VMC training (Methods, ansatz optimisation: Adam with
 * decoupled weight decay after Loshchilov and Hutter, the total energy as
 * the loss, Eq. trainig for its gradient):
 *   m <- b1 m + (1 - b1) g;  v <- b2 v + (1 - b2) g^2;
 *   theta <- theta - lr (m / (1 - b1^t) / (sqrt(v / (1 - b2^t)) + eps)
 *                        + weight_decay theta).
 * theta, grad, m, v: n float64 DEVICE buffers (m and v start at zero and
 * are updated in place); t >= 1 is the step count.  Asynchronous on the
 * stream; PN_EINVAL for host buffers or out-of-range hyperparameters. */
int pn_adamw_step(double* theta, const double* grad, double* m, double* v,
                  int64_t n, double lr, double beta1, double beta2, double eps,
                  double weight_decay, int64_t t, void* stream);

typedef struct pn_server_cfg {
  size_t hbm_budget_bytes;   /* total device memory the server may hold */
  int n_slots;               /* concurrent jobs (one stream each)       */
  int chunk_walkers;         /* walkers per workspace chunk per job     */
  int debug_fail_nth;        /* test hook: the n-th admitted job fails on
                                the host before it launches anything
                                (result status PN_EDEVICE); 0 = off     */
} pn_server_cfg;

enum { PN_JOB_ELOC = 0, PN_JOB_SWEEP = 1, PN_JOB_SCAN = 2 };

typedef struct pn_job {
  int kind;          /* PN_JOB_ELOC: E_loc of the walkers; PN_JOB_SWEEP:
                        n_steps Metropolis steps, then E_loc;
                        PN_JOB_SCAN: E_loc at W points of a line scan
                        (pn_eval_line_scan) of the base configuration
                        r_init [N][3] (required), r_out unused           */
  int W;
  int n_steps;
  double sigma;
  uint64_t seed;
  const double* r_init;  /* [W][N][3] host or device, or NULL -> pn_init_walkers */
  double* eloc_out;      /* [W] host or device, or NULL                 */
  double* r_out;         /* [W][N][3] host or device, or NULL           */
  int scan_electron;     /* PN_JOB_SCAN: the moving electron            */
  double scan_dir[3];    /* PN_JOB_SCAN: direction of the line          */
  double scan_t0, scan_t1;  /* PN_JOB_SCAN: first and last parameter  */
} pn_job;

typedef struct pn_result {
  int status;            /* PN_OK, PN_ECANCELLED or an error code        */
  int W;
  double e_mean;         /* mean E_loc over finite walkers              */
  double e_stderr;       /* standard error of the mean                  */
  double accept_rate;    /* sweeps only                                 */
  int64_t n_nonfinite;   /* walkers with status != PN_WALKER_OK        */
  double queue_ms;       /* submit -> admission                         */
  double run_ms;         /* admission -> completion                     */
  double dev_start_ms;   /* the job's first device work, ms after the   */
  double dev_end_ms;     /*   server's creation; and its last (CUDA
                            events on the job's stream; 0 on failure)   */
  int64_t n_guarded;     /* walkers the mixed local-energy guard
                            re-evaluated in float64 (PN_OPT_GUARD)      */
} pn_result;

int pn_server_create(const pn_server_cfg* cfg, pn_server_t* out);
/* Stops the loop after the running jobs finish; queued jobs are cancelled. */
int pn_server_destroy(pn_server_t srv);
/* Queue a job.  PN_EBUDGET at once if its footprint can never fit. */
int pn_submit(pn_server_t srv, pn_system_t sys, const pn_job* job, uint64_t* job_id);
/* PN_OK with *res filled once done (the job is then forgotten; res->status
 * says how it ended: PN_OK, PN_ECANCELLED or an error), PN_ENOTREADY if
 * timeout_us == 0 and not done, PN_ETIMEOUT if it did not finish within
 * timeout_us (> 0), PN_EINVAL for an unknown id.  A negative timeout waits
 * until the job ends. */
int pn_poll(pn_server_t srv, uint64_t job_id, pn_result* res, int64_t timeout_us);
/* Cancel a queued job (PN_OK) -- running jobs complete (PN_ENOTREADY). */
int pn_cancel(pn_server_t srv, uint64_t job_id);
/* Device bytes a job of this size would hold. */
size_t pn_job_footprint(pn_system_t sys, int W, int chunk_walkers);

/* Self-test of the tensor-core linear layer used by the mixed path (no
 * counterpart in the paper): Y (=|+=) X W + b on device float32 buffers,
 * X [rows][K] (row stride ldx), W [K][Nout] (row stride ldw), Y [rows][Nout]
 * (row stride ldy), bias added on rows with row % T == 0; Nout <= 256.
 * Runs on `stream` and synchronises it; PN_ETIMEOUT if the kernel's bounded
 * wait for the tensor cores expired. */
int pn_test_linear_tc(const float* X, int ldx, const float* W, int ldw,
                      const float* b, float* Y, int ldy, int rows, int K,
                      int Nout, int T, int accumulate, void* stream);

/* ---------------------------------------------------------------------
 * Measurement hooks (no counterpart in the paper).
 * pn_launch_count: kernels this library has launched since load.
 * pn_profile_kernel: time every later launch of the kernel class `name`
 *   (NULL or "" stops) with a CUDA event pair on the launch's own stream;
 *   clears earlier records.
 * pn_profile_read: synchronises those events and returns how many launches
 *   were timed and their summed duration in ms.
 * pn_profile_work: the algorithmic work of those launches, summed as their
 *   launch sites report it -- floating-point operations (a multiply-add
 *   counts 2) for compute kernels, bytes that must cross HBM for the
 *   message kernels; 0 for kernel classes that report none.
 * pn_profile_bytes: the bytes those launches must move through HBM at
 *   least (inputs read and outputs written once), summed as the launch sites
 *   that know them report it (the linear maps); 0 for the others.
 * pn_measure_peak: the issue-rate ceiling of a CUDA-core unit on the
 *   current device, measured by this library's own kernel (eight
 *   independent multiply-add chains per thread, 8 blocks of 256 threads per
 *   SM, best of two timed launches after one warm-up): kind 0 float32 FMA,
 *   1 float64 FMA; *tflops in TFLOP/s.  Synchronises `stream`; changes no
 *   device setting.
 */
unsigned long long pn_launch_count(void);
int pn_profile_kernel(const char* name);
int pn_profile_read(int64_t* count, double* total_ms);
int pn_profile_work(double* work);
int pn_profile_bytes(double* bytes);
int pn_measure_peak(int kind, double* tflops, void* stream);

const char* pn_last_error(void);

#ifdef __cplusplus
}
#endif
#endif /* PAULINET_H */
