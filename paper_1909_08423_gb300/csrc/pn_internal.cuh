// Internal declarations shared by the translation units of libpaulinet.so.
#pragma once

#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/paulinet.h"

#define PN_LMAX PN_MAX_LAYERS

// ---------------------------------------------------------------- errors
void pn_set_error(const char* fmt, ...);

#define PN_CUDA(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess) {                                                 \
      pn_set_error("%s:%d %s: %s", __FILE__, __LINE__, #call,                \
                   cudaGetErrorString(e_));                                  \
      return PN_EDEVICE;                                                     \
    }                                                                        \
  } while (0)

// Launch bookkeeping (profile.cu): count, and optional event timing of one
// kernel class.  PN_LAUNCH(name, stream, launch-expression).  Every launch
// also sits in an NVTX range named by its class (a no-op unless a tool that
// records NVTX is attached).
void pn_prof_begin(const char* name, cudaStream_t st);
void pn_note_launch(const char* name, cudaStream_t st);
// Algorithmic work of the launch just made (FLOPs, or bytes for kernels
// bound by memory traffic), summed while `name` is the timed class.
void pn_prof_work(const char* name, double work);
// Bytes the launch just made must move through HBM at least (its inputs
// read and outputs written once), for launch sites that know them.
void pn_prof_bytes(const char* name, double bytes);
#define PN_CHECK_LAUNCH() PN_CUDA(cudaGetLastError())
#define PN_LAUNCH(name, st, ...)        \
  do {                                  \
    nvtxRangePushA(name);               \
    pn_prof_begin(name, st);            \
    __VA_ARGS__;                        \
    pn_note_launch(name, st);           \
    nvtxRangePop();                     \
    PN_CHECK_LAUNCH();                  \
  } while (0)
// The same with the launch's algorithmic work (see pn_prof_work) and, for
// PN_LAUNCH_WB, its algorithmic bytes (pn_prof_bytes).
#define PN_LAUNCH_W(name, st, work, ...) \
  do {                                   \
    nvtxRangePushA(name);                \
    pn_prof_begin(name, st);             \
    __VA_ARGS__;                         \
    pn_note_launch(name, st);            \
    pn_prof_work(name, (double)(work));  \
    nvtxRangePop();                      \
    PN_CHECK_LAUNCH();                   \
  } while (0)
#define PN_LAUNCH_WB(name, st, work, bytes, ...) \
  do {                                           \
    nvtxRangePushA(name);                        \
    pn_prof_begin(name, st);                     \
    __VA_ARGS__;                                 \
    pn_note_launch(name, st);                    \
    pn_prof_work(name, (double)(work));          \
    pn_prof_bytes(name, (double)(bytes));        \
    nvtxRangePop();                              \
    PN_CHECK_LAUNCH();                           \
  } while (0)

// Allow a kernel every dynamic shared-memory size up to the device's
// opt-in limit.  Every caller sets the same value, so host threads that
// launch one kernel with different sizes (serving slots of different
// systems) cannot lower the limit under one another's launch.
template <typename F>
inline cudaError_t pn_allow_max_smem(F* f) {
  int dev = 0, v = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&v, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (cudaError_t e = cudaFuncGetAttributes(&fa, f)) return e;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, v - (int)fa.sharedSizeBytes);
}

// ------------------------------------------------------------- parameters
// Offsets (in elements) of every tensor inside the flat parameter vector.
struct NetOff {
  int64_t x0, Y;
  int64_t hW[PN_LMAX], hb[PN_LMAX];
  int64_t W1[PN_LMAX][3], b1[PN_LMAX][3], W2[PN_LMAX][3], b2[PN_LMAX][3];
  int64_t GW[PN_LMAX][3], Gb[PN_LMAX][3];
  int64_t eW[3], eb[3], kW[3], kb[3];
  int64_t total;
};
NetOff pn_net_offsets(int D, int Zd, int K, int L, int M, int n_orb);

// ------------------------------------------------- device view of a system
// Everything a kernel needs, passed by value.  Pointers are device memory.
struct DevSys {
  int N, n_up, n_dn, M, n_b, n_orb, n_det, n_shells;
  int D, Zd, K, L, Hw;
  int Pee;          // unordered electron pairs N(N-1)/2
  int Pen;          // electron-nucleus pairs N*M
  int Ppair;        // Pee + Pen
  double r_c;
  int use_cusp, use_gamma;
  double Vnn;
  const double* Z;        // [M]
  const double* R;        // [M*3]
  const int* sh_center;   // [n_shells]
  const int* sh_l;
  const int* sh_nprim;
  const int* sh_poff;     // first primitive
  const int* sh_boff;     // first basis function
  const double* pexp;
  const double* pcoef;
  const double* mo;       // [n_b][n_orb]
  const int* occ;         // [n_det][N]: up orbitals then down orbitals
  const double* ci;       // [n_det]
  const double* cusp_rc;  // [M]
  const int* cusp_on;     // [M][n_orb]
  const double* cusp_C;   // [M][n_orb]
  const double* cusp_s;   // [M][n_orb]
  const double* cusp_a;   // [M][n_orb][5]
  const double* feat_mu;  // [K]
  const double* feat_isig2;  // [K] 1/sigma^2
  const float* feat_mu32;    // [K] float copies for float32 paths
  const float* feat_isig2_32;
  // float copies of the orbital tables for the mixed sampler
  const float* R32;
  const float* pexp32;
  const float* pcoef32;
  const float* mo32;
  const float* cusp_rc32;
  const float* cusp_C32;
  const float* cusp_s32;
  const float* cusp_a32;
  const int* nuc;         // [N] nucleus each electron starts near (walker init)
  const int* ch_pairs;    // [Ppair] pair indices grouped by filter channel
  int ch_off[4];          // channel c owns ch_pairs[ch_off[c] .. ch_off[c+1])
  const int* ch_pos;      // [Ppair] position of each pair inside its channel's list
  // Table of the determinant expansion relative to determinant 0 (jet
  // determinants by the table method, slater_table.cu); null when a
  // determinant is not reachable from determinant 0 by at most
  // PN_TAB_KMAX replacements or a block exceeds PN_TAB_NMAX / PN_TAB_VMAX.
  // Layout: per spin {n_virt, virtual orbitals [PN_MAX_ORBITALS]}, then per
  // (determinant, spin) a record {k, sign, holes[KMAX], particles[KMAX]}
  // (holes: positions in determinant 0's list; particles: indices into the
  // spin's virtual orbitals).
  const int* xtab;
  int tab_wstride;        // doubles of shared memory per warp of the table kernel
  int tab_nv[2];          // virtual orbitals per spin
  int tab_k3[2];          // sum over determinants of k^3 per spin
  int guard_probe;        // second evaluation of the guard: 0 heads on the other unit, 1 perturbed jets,
                          // 2 perturbed jets at the relative and the term scale
  int msg_per_row;        // 1: jet messages by the per-row kernel even where the staged one applies
  int no_table;           // 1: jet determinants block by block even where a table exists;
                          // 2: the table kernel with every walker on its direct fallback
  int fused_sampler;      // 1: Metropolis through the fused tile kernel when it fits
  int tensor_cores;       // mask of float32 linear-layer groups on tcgen05 (split bf16)
  int lin_f32x2;          // 1: float64 linear maps as float32 pairs (the guard's re-evaluation)
  int* dev_err;           // device word: set when a bounded wait expired
};

#define PN_TAB_NMAX 8
#define PN_TAB_VMAX 8
#define PN_TAB_KMAX 4
#define PN_TAB_REC (2 + 2 * PN_TAB_KMAX)

// Determinants by the table method (slater_table.cu; value or jet mode):
// PN_ENOTREADY when the system has no table or the warp's matrices do not fit.
template <typename R>
int pn_slater_table_launch(const DevSys& s, const double* phi, const R* F, int Wn, int T, int jet, double* det,
                           cudaStream_t st);
double pn_slater_table_flops(const DevSys& s, int jet);

// Pair indexing: unordered electron pair (a<b) -> a*N - a*(a+1)/2 + (b-a-1)
__host__ __device__ inline int pn_pair_index(int a, int b, int N) {
  return a * N - a * (a + 1) / 2 + (b - a - 1);
}

// ------------------------------------------------------------- workspace
// One chunk of walkers' intermediates.  T = jet rows (1 or 3N+2).
template <typename R>
struct Work {
  int Wc;                 // walkers per chunk
  int T;                  // jet rows the buffers were sized for
  double* r;              // [Wc][N][3] staging of host positions
  double* geo;            // [Wc][Ppair][4]  (d, unit vector)
  double* phi;            // [Wc][N][n_orb][5] value, grad, lap
  R* efeat;               // [Wc][Ppair][3][K] distance features e, e', e''
  R* wjet;                // [Wc][Ppair][3][Zd]
  R* X;                   // [Wc][N][T][D]
  R* H;                   // [Wc][N][T][max(Zd, D)]
  R* Zb;                  // [Wc][N][T][max(3 Zd, D)]
  R* Xs;                  // [Wc][T][D]
  R* As;                  // [Wc][T][D]
  R* Bs;                  // [Wc][T][D]
  R* F;                   // [Wc][N][T][n_orb]
  R* Jj;                  // [Wc][T]
  double* det;            // [Wc][n_det][2][3 + 3N] : ld, sign, lap, grad[3N]
  double* out_logabs;     // [Wc]
  double* out_sign;       // [Wc]
  double* out_eloc;       // [Wc]
  double* out_grad;       // [Wc][3N]  grad_r ln|psi| of the jet pass
  int* out_status;        // [Wc]
  unsigned long long* n_acc;  // [1]
  double* r_prop;         // [Wc][N][3]
  double* lp_prop;        // [Wc]
  int ldH, ldZ;           // row strides of H and Zb
  char* end;              // one past the last carved byte
};

size_t pn_work_bytes(const DevSys& s, int Wc, int T, int elem);

// Weight blocks of the fused sampler in the order it consumes them: per
// layer h, (W1, W2) for the three filter channels, stacked receiving maps;
// then kappa 1..3 and eta 1..3.  Each block starts 16-byte aligned in a
// packed copy of the weights so that it can be bulk-copied (TMA) into
// shared memory.
constexpr int PN_MAX_STAGES = 8 * PN_MAX_LAYERS + 6;
struct StageTab {
  int n;                        // stages per Metropolis step
  int max_bytes;                // largest block
  int64_t off[PN_MAX_STAGES];   // element offset in the packed weights
  int bytes[PN_MAX_STAGES];     // block size in bytes (multiple of 16)
};

// Weight blocks of the tensor-core sampler, in consumption order: per layer
// h, then for every non-empty filter channel (W1, W2, receiving-map slice);
// then kappa 1..3 and eta 1..3.  Each block is stored as three bf16 pieces
// of the transposed weight (rows = outputs padded to 16, columns = inputs)
// in the canonical K-major tile layout of tcgen05 (8 x 16-byte core
// matrices), so that one bulk copy lands it ready for the MMA.
constexpr int PN_MAX_TC_STAGES = 10 * PN_MAX_LAYERS + 6;  // h + 3 x (W1, W2, G) per layer, 6 head maps
struct TcStages {
  int n;                          // stages per Metropolis step (0: not eligible)
  int max_bytes;
  int64_t off[PN_MAX_TC_STAGES];  // bf16 element offset in the packed blocks
  int bytes[PN_MAX_TC_STAGES];    // bytes (three pieces)
  int K[PN_MAX_TC_STAGES];        // inputs
  int Np[PN_MAX_TC_STAGES];       // outputs padded to 16
};

// Per-precision parameters on the device.
template <typename R>
struct DevNet {
  const R* p;      // flat parameter vector in R
  const float* p2; // float64 networks: the same as (hi, lo) float pairs (float32-pair arithmetic); else null
  const R* Gcat;   // [L][3 Zd][D]  same, anti, nuc receiving maps stacked
  const R* Gb;     // [L][D]        sum of the three receiving biases
  const R* Gbx0;   // [D]           first layer's summed bias + x^(0)
  const R* wpack;  // sampler weight blocks, 16-byte aligned (see StageTab)
  NetOff off;
  StageTab stab;
  const unsigned short* tcpack;  // tensor-core sampler blocks (float path only)
  const TcStages* tcst;          // their table, in device memory
  int tc_n, tc_max_bytes;        // host copies of its size fields
};

// Guard of the mixed-precision local energy.  The float32 network's
// rounding reaches E_loc through the determinants and the squared gradient,
// and a few walkers per ten thousand amplify it beyond 1e-4 Ha; no cheap
// per-walker quantity predicts which.  So every mixed jet chunk is
// evaluated twice: the heads run again on the other unit (tensor cores
// instead of CUDA cores or back), which changes their rounding, and the
// determinants and E_loc are formed from the second heads.  Walkers whose two
// energies differ by more than tau (or are not finite) are evaluated again
// in float64 and take the float64 results.  The float64 pass runs on its own
// workspace of `cap` walkers.
struct Guard {
  double tau;            // hartree; <= 0 turns the guard off
  int cap;               // walkers per float64 re-evaluation
  Work<double> w64;      // float64 jet workspace for cap walkers
  DevNet<double> net64;  // float64 parameters of the same system
  double* e_probe;       // [Wc] E_loc of the second evaluation
  int* list;             // [Wc] flagged walkers of the chunk
  int* pend;             // [cap] flagged walkers of earlier chunks of the call, global indices
  int* count;            // [2] device: flagged walkers, walkers re-evaluated so far
  int64_t* n_total;      // [1] device: walkers re-evaluated since the last read
};
size_t pn_guard_bytes(const DevSys& s, int Wc, int cap);
Guard pn_carve_guard(const DevSys& s, int Wc, int cap, void* base);

struct pn_system_s {
  DevSys ds;
  Guard guard;              // mixed handles: local-energy guard (tau 0: off)
  void* guard_mem;
  NetOff off;
  int precision;
  int no_jastrow, no_backflow;  // ablation variants: head removed
  int drift_mode;               // grad_r ln|psi| for Langevin moves: 0 jet pass, 1 reverse mode
  int Wc;
  int Tjet;
  // device allocations
  std::vector<void*> allocs;
  double* p64;
  float* p32;
  float* p2_64;  // p64 as (hi, lo) float pairs
  double* Gcat64;
  double* Gb64;
  float* Gcat32;
  float* Gb32;
  double* Gbx0_64;
  float* Gbx0_32;
  void* work_mem;
  size_t work_bytes;
  StageTab stab64, stab32;  // packed sampler weights per precision
  TcStages tcst;            // tensor-core sampler weight blocks
  TcStages* tcst_dev;       // the same table in device memory
  unsigned short* tcpack;   // [tcst total] bf16 pieces
  double* wpack64;
  float* wpack32;
  void* tape_mem;          // backward tape (grown on demand)
  size_t tape_bytes;
  Work<double> w64;
  Work<float> w32;
  // host copies
  std::vector<double> h_params;
  int device;
};

// Carve a workspace out of one allocation.
template <typename R>
Work<R> pn_carve_work(const DevSys& s, int Wc, int T, void* base);

// ----------------------------------------------------------- forward path
// mode: 0 value only (T = 1), 1 jet (T = 3N + 2)
template <typename R>
int pn_forward_chunk(const DevSys& s, const DevNet<R>& net, Work<R>& w,
                     const double* r, int Wn, int jet, cudaStream_t st);

template <typename R>
DevNet<R> pn_devnet(pn_system_s* sys);

// Tensor-core linear layer (tc_gemm.cu).
bool pn_tc_supported(int Nout);
int pn_linear_tc(const float* X, int ldx, const float* W, int ldw, const float* b, float* Y, int ldy, int rows, int K,
                 int Nout, int T, int acc, int* err, cudaStream_t st,
                 int absval = 0);


// Chunked drivers over an explicit workspace (used by the C ABI with the
// handle's workspace and by the serving loop with per-job workspaces).
// g (mixed jet passes only; may be null) guards the local energies.
template <typename R>
int pn_run_eval(const DevSys& ds, const DevNet<R>& net, Work<R>& w, int Wc, const double* r, int W, int jet,
                double* eloc, double* logabs, double* sign, int* status, cudaStream_t st,
                const Guard* g = nullptr);
// The second evaluation of a guarded chunk: heads on the other unit,
// determinants, E_loc into e_probe (w.X, w.phi and w.geo hold the chunk's
// first pass; w's other outputs are left as the first pass wrote them).
// The guard's perturbations (guard_probe.cu): every element of A times
// (1 +- eta); and y += +-(eta_rel |y| + eta_abs sum_k |x_k| |W_kn|) over the
// output Y = X W of a linear map (X rows x Kd, W Kd x Nout).
int pn_perturb_rel(float* A, size_t n, float eta, cudaStream_t st);
int pn_perturb_abs(const float* X, int ldx, const float* W, int ldw, float* Y, int ldy, size_t rows, int Kd, int Nout,
                   float eta_rel, float eta_abs, cudaStream_t st);
// The same with the term scale formed by the tensor-core map in
// absolute-value mode into scratch (rows x Nout floats); PN_ENOTREADY when
// scratch is too small or the map does not fit.
int pn_perturb_abs_tc(const float* X, int ldx, const float* W, int ldw, float* Y, int ldy, size_t rows, int Kd,
                      int Nout, float eta_rel, float eta_abs, float* scratch, size_t scratch_floats, int* err,
                      cudaStream_t st);
int pn_probe_heads_chunk(const DevSys& s, const DevNet<float>& net, Work<float>& w, int Wn, double* e_probe,
                         cudaStream_t st);
template <typename R>
int pn_run_metropolis(const DevSys& ds, const DevNet<R>& net, Work<R>& w, int Wc, double* r, double* logabs, int W,
                      int n_steps, double sigma, unsigned long long seed, unsigned long long step0, int64_t* n_accept,
                      cudaStream_t st);
template <typename R>
int pn_run_line_scan(const DevSys& ds, const DevNet<R>& net, Work<R>& w, int Wc, const double* r0, int e,
                     const double dir[3], double t0, double t1, int npts, double* eloc, double* logabs, double* sign,
                     int* status, cudaStream_t st);
int pn_run_init_walkers(const DevSys& ds, double* r, int W, unsigned long long seed, cudaStream_t st);
// Tensor-core sampler (sampler_tc.cu): PN_ENOTREADY if the system's tiles do not fit.
int pn_run_metropolis_tc(const DevSys& s, const DevNet<float>& net, double* r, double* lp, int W, unsigned walker0,
                         int n_steps, double sigma, unsigned long long seed, unsigned long long step0,
                         unsigned long long* n_acc, cudaStream_t st);
// Fused sampler (sampler.cu): PN_ENOTREADY if a tile does not fit.
template <typename R>
int pn_run_metropolis_fused(const DevSys& s, const DevNet<R>& net, double* r, double* lp, int W, unsigned walker0,
                            int n_steps, double sigma, unsigned long long seed, unsigned long long step0,
                            unsigned long long* n_acc, cudaStream_t st);

// ln|psi| and grad_r ln|psi| of Wn <= max(Wc, Wn) walkers at device
// positions r by reverse mode (backward.cu), on the system's tape (grown on
// demand); logabs [Wn] and grad [Wn][N][3] are device buffers.
template <typename R>
int pn_drift_reverse(pn_system_s* sys, const double* r, int Wn, double* logabs, double* grad, cudaStream_t st);

// Host/device pointer check.
bool pn_is_device_ptr(const void* p);

int pn_get_stream_device(cudaStream_t st);
