// System set-up: validation, host precompute of the nuclear cusp splice,
// parameter packing, device upload and workspace sizing.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include <algorithm>
#include <string>
#include <vector>

#include "pn_internal.cuh"

static thread_local std::string g_err;

void pn_set_error(const char* fmt, ...) {
  char buf[1024];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
}

extern "C" const char* pn_last_error(void) { return g_err.c_str(); }

bool pn_is_device_ptr(const void* p) {
  if (!p) return false;
  cudaPointerAttributes a;
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return a.type == cudaMemoryTypeDevice || a.type == cudaMemoryTypeManaged;
}

// ------------------------------------------------------------ parameters
NetOff pn_net_offsets(int D, int Zd, int K, int L, int M, int n_orb) {
  NetOff o;
  memset(&o, 0, sizeof o);
  int Hw = std::max(K, Zd);
  int64_t c = 0;
  o.x0 = c; c += D;
  o.Y = c; c += (int64_t)M * Zd;
  for (int n = 0; n < L; ++n) {
    o.hW[n] = c; c += (int64_t)D * Zd;
    o.hb[n] = c; c += Zd;
    for (int ch = 0; ch < 3; ++ch) {
      o.W1[n][ch] = c; c += (int64_t)K * Hw;
      o.b1[n][ch] = c; c += Hw;
      o.W2[n][ch] = c; c += (int64_t)Hw * Zd;
      o.b2[n][ch] = c; c += Zd;
    }
    for (int ch = 0; ch < 3; ++ch) {
      o.GW[n][ch] = c; c += (int64_t)Zd * D;
      o.Gb[n][ch] = c; c += D;
    }
  }
  const int outs[3] = {D, D, 1};
  for (int k = 0; k < 3; ++k) {
    o.eW[k] = c; c += (int64_t)D * outs[k];
    o.eb[k] = c; c += outs[k];
  }
  const int kouts[3] = {D, D, n_orb};
  for (int k = 0; k < 3; ++k) {
    o.kW[k] = c; c += (int64_t)D * kouts[k];
    o.kb[k] = c; c += kouts[k];
  }
  o.total = c;
  return o;
}

extern "C" int64_t pn_num_params_for(int D, int Zd, int K, int L, int M, int n_orb) {
  if (L < 0 || L > PN_LMAX) return -1;
  return pn_net_offsets(D, Zd, K, L, M, n_orb).total;
}

// -------------------------------------------------------- host basis eval
namespace {

int ncart(int l) { return l <= 0 ? 1 : (l == 1 ? 3 : 6); }

const int CART2[6][3] = {{2, 0, 0}, {1, 1, 0}, {1, 0, 1}, {0, 2, 0}, {0, 1, 1}, {0, 0, 2}};
const int CART1[3][3] = {{1, 0, 0}, {0, 1, 0}, {0, 0, 1}};

void cart_exps(int l, int c, int e[3]) {
  if (l <= 0) { e[0] = e[1] = e[2] = 0; return; }
  const int* s = (l == 1) ? CART1[c] : CART2[c];
  e[0] = s[0]; e[1] = s[1]; e[2] = s[2];
}

struct HostSys {
  int M, N, n_up, n_dn, n_orb, n_b, n_det, n_shells;
  std::vector<double> Z, R;
  std::vector<int> sc, sl, sn, spo, sbo;
  std::vector<double> pe, pc, mo;
};

// Uncorrected orbital values at a point.
void host_orbitals(const HostSys& h, const double* p, std::vector<double>& phi) {
  phi.assign(h.n_orb, 0.0);
  for (int s = 0; s < h.n_shells; ++s) {
    const double* Rc = &h.R[3 * h.sc[s]];
    double v[3] = {p[0] - Rc[0], p[1] - Rc[1], p[2] - Rc[2]};
    double r2 = v[0] * v[0] + v[1] * v[1] + v[2] * v[2];
    int l = h.sl[s];
    if (l == -1) {
      double val = h.pc[h.spo[s]] * exp(-h.pe[h.spo[s]] * sqrt(r2));
      for (int mu = 0; mu < h.n_orb; ++mu) phi[mu] += h.mo[(size_t)h.sbo[s] * h.n_orb + mu] * val;
      continue;
    }
    double rad = 0;
    for (int k = 0; k < h.sn[s]; ++k) rad += h.pc[h.spo[s] + k] * exp(-h.pe[h.spo[s] + k] * r2);
    for (int c = 0; c < ncart(l); ++c) {
      int e[3];
      cart_exps(l, c, e);
      double pv = 1;
      for (int a = 0; a < 3; ++a)
        for (int q = 0; q < e[a]; ++q) pv *= v[a];
      for (int mu = 0; mu < h.n_orb; ++mu)
        phi[mu] += h.mo[(size_t)(h.sbo[s] + c) * h.n_orb + mu] * pv * rad;
    }
  }
}

// Radial s part of orbital mu on nucleus I and its two radial derivatives.
void host_s_part(const HostSys& h, int I, int mu, double r, double* f, double* f1, double* f2) {
  *f = *f1 = *f2 = 0;
  for (int s = 0; s < h.n_shells; ++s) {
    if (h.sl[s] != 0 || h.sc[s] != I) continue;
    double c = h.mo[(size_t)h.sbo[s] * h.n_orb + mu];
    for (int k = 0; k < h.sn[s]; ++k) {
      double a = h.pe[h.spo[s] + k];
      double d = h.pc[h.spo[s] + k] * c;
      double e = exp(-a * r * r);
      *f += d * e;
      *f1 += -2.0 * a * r * d * e;
      *f2 += (4.0 * a * a * r * r - 2.0 * a) * d * e;
    }
  }
}

bool solve3(double A[3][3], double b[3], double x[3]) {
  // Gaussian elimination with partial pivoting on a 3x3 system.
  double M[3][4];
  for (int i = 0; i < 3; ++i) {
    for (int j = 0; j < 3; ++j) M[i][j] = A[i][j];
    M[i][3] = b[i];
  }
  for (int c = 0; c < 3; ++c) {
    int best = c;
    for (int r = c + 1; r < 3; ++r)
      if (fabs(M[r][c]) > fabs(M[best][c])) best = r;
    if (M[best][c] == 0.0) return false;
    if (best != c)
      for (int j = 0; j < 4; ++j) std::swap(M[c][j], M[best][j]);
    for (int r = c + 1; r < 3; ++r) {
      double f = M[r][c] / M[c][c];
      for (int j = c; j < 4; ++j) M[r][j] -= f * M[c][j];
    }
  }
  for (int i = 2; i >= 0; --i) {
    double acc = M[i][3];
    for (int j = i + 1; j < 3; ++j) acc -= M[i][j] * x[j];
    x[i] = acc / M[i][i];
  }
  return true;
}

template <typename T>
T* dev_upload(pn_system_s* s, const T* h, size_t n, int* err) {
  if (n == 0) n = 1;
  void* p = nullptr;
  if (cudaMalloc(&p, n * sizeof(T)) != cudaSuccess) {
    cudaGetLastError();
    *err = PN_ENOMEM;
    return nullptr;
  }
  s->allocs.push_back(p);
  if (h && cudaMemcpy(p, h, n * sizeof(T), cudaMemcpyHostToDevice) != cudaSuccess) {
    *err = PN_EDEVICE;
    return nullptr;
  }
  return (T*)p;
}

void free_all(pn_system_s* s) {
  for (void* p : s->allocs) cudaFree(p);
  s->allocs.clear();
  if (s->work_mem) cudaFree(s->work_mem);
  s->work_mem = nullptr;
  if (s->tape_mem) cudaFree(s->tape_mem);
  s->tape_mem = nullptr;
  if (s->guard_mem) cudaFree(s->guard_mem);
  s->guard_mem = nullptr;
}

}  // namespace

// ------------------------------------------------------------- workspace
static size_t align_up(size_t x) { return (x + 255) & ~(size_t)255; }

size_t pn_work_bytes(const DevSys& s, int Wc, int T, int elem) {
  size_t W = Wc, N = s.N;
  size_t ldH = std::max(s.Zd, s.D), ldZ = std::max(3 * s.Zd, s.D);
  size_t b = 0;
  b += align_up(W * N * 3 * 8);                      // r
  b += align_up(W * s.Ppair * 4 * 8);                // geo
  b += align_up(W * N * s.n_orb * 5 * 8);            // phi
  b += align_up(W * s.Ppair * 3 * s.K * elem);       // efeat (lives after wjet)
  b += align_up(W * s.Ppair * 3 * s.Zd * elem);      // wjet
  b += align_up(W * N * T * s.D * elem);             // X
  b += align_up(W * N * T * ldH * elem);             // H
  b += align_up(W * N * T * ldZ * elem);             // Zb
  b += 3 * align_up(W * T * s.D * elem);             // Xs, As, Bs
  b += align_up(W * N * T * s.n_orb * elem);         // F
  b += align_up(W * T * elem);                       // Jj
  b += align_up(W * s.n_det * 2 * (3 + 3 * N) * 8);  // det
  b += 3 * align_up(W * 8) + align_up(W * 4);        // outputs
  b += align_up(W * N * 3 * 8);                      // grad ln|psi|
  b += align_up(8);                                  // n_acc
  b += align_up(W * N * 3 * 8) + align_up(W * 8);    // proposals
  return b;
}

template <typename R>
Work<R> pn_carve_work(const DevSys& s, int Wc, int T, void* base) {
  Work<R> w;
  char* p = (char*)base;
  size_t W = Wc, N = s.N;
  size_t ldH = std::max(s.Zd, s.D), ldZ = std::max(3 * s.Zd, s.D);
  size_t elem = sizeof(R);
  auto take = [&](size_t bytes) { char* q = p; p += align_up(bytes); return (void*)q; };
  w.Wc = Wc;
  w.T = T;
  w.r = (double*)take(W * N * 3 * 8);
  w.geo = (double*)take(W * s.Ppair * 4 * 8);
  w.phi = (double*)take(W * N * s.n_orb * 5 * 8);
  w.efeat = (R*)take(W * s.Ppair * 3 * s.K * elem);
  w.wjet = (R*)take(W * s.Ppair * 3 * s.Zd * elem);
  w.X = (R*)take(W * N * T * s.D * elem);
  w.H = (R*)take(W * N * T * ldH * elem);
  w.Zb = (R*)take(W * N * T * ldZ * elem);
  w.Xs = (R*)take(W * T * s.D * elem);
  w.As = (R*)take(W * T * s.D * elem);
  w.Bs = (R*)take(W * T * s.D * elem);
  w.F = (R*)take(W * N * T * s.n_orb * elem);
  w.Jj = (R*)take(W * T * elem);
  w.det = (double*)take(W * s.n_det * 2 * (3 + 3 * N) * 8);
  w.out_logabs = (double*)take(W * 8);
  w.out_sign = (double*)take(W * 8);
  w.out_eloc = (double*)take(W * 8);
  w.out_status = (int*)take(W * 4);
  w.out_grad = (double*)take(W * N * 3 * 8);
  w.n_acc = (unsigned long long*)take(8);
  w.r_prop = (double*)take(W * N * 3 * 8);
  w.lp_prop = (double*)take(W * 8);
  w.ldH = (int)ldH;
  w.ldZ = (int)ldZ;
  w.end = p;
  return w;
}
template Work<double> pn_carve_work<double>(const DevSys&, int, int, void*);
template Work<float> pn_carve_work<float>(const DevSys&, int, int, void*);

// Guard of the mixed local energy: a float64 jet workspace for cap walkers,
// then the per-chunk probe energies, flag list and counters.
size_t pn_guard_bytes(const DevSys& s, int Wc, int cap) {
  return align_up(pn_work_bytes(s, cap, 3 * s.N + 2, 8)) + align_up((size_t)Wc * 8) + align_up((size_t)Wc * 4) +
         align_up((size_t)cap * 4) + align_up(2 * sizeof(int)) + align_up(8);
}

Guard pn_carve_guard(const DevSys& s, int Wc, int cap, void* base) {
  Guard g;
  g.tau = 0;
  g.cap = cap;
  char* p = (char*)base;
  g.w64 = pn_carve_work<double>(s, cap, 3 * s.N + 2, p);
  p += align_up(pn_work_bytes(s, cap, 3 * s.N + 2, 8));
  g.e_probe = (double*)p;
  p += align_up((size_t)Wc * 8);
  g.list = (int*)p;
  p += align_up((size_t)Wc * 4);
  g.pend = (int*)p;
  p += align_up((size_t)cap * 4);
  g.count = (int*)p;
  p += align_up(2 * sizeof(int));
  g.n_total = (int64_t*)p;
  return g;
}

// ----------------------------------------------------------- parameters
static int upload_params(pn_system_s* s, const double* hp_user) {
  const DevSys& d = s->ds;
  const NetOff& o = s->off;
  s->h_params.assign(hp_user, hp_user + o.total);
  // ablation variants: the removed head's last map is zero, so that every
  // kernel computes J = 0 or f = 1 exactly
  std::vector<double> masked(hp_user, hp_user + o.total);
  if (s->no_jastrow) std::fill(masked.begin() + o.eW[2], masked.begin() + o.eb[2] + 1, 0.0);
  if (s->no_backflow) std::fill(masked.begin() + o.kW[2], masked.begin() + o.kb[2] + d.n_orb, 0.0);
  const double* hp = masked.data();
  PN_CUDA(cudaMemcpy(s->p64, hp, o.total * 8, cudaMemcpyHostToDevice));
  {
    // hi = the nearest float, lo = the nearest float of the rest
    std::vector<float> p2(2 * (size_t)o.total);
    for (int64_t k = 0; k < o.total; ++k) {
      const float hi = (float)hp[k];
      p2[2 * k] = hi;
      p2[2 * k + 1] = (float)(hp[k] - (double)hi);
    }
    PN_CUDA(cudaMemcpy(s->p2_64, p2.data(), p2.size() * 4, cudaMemcpyHostToDevice));
  }
  std::vector<float> p32(hp, hp + o.total);
  PN_CUDA(cudaMemcpy(s->p32, p32.data(), o.total * 4, cudaMemcpyHostToDevice));
  // stacked receiving maps and summed biases per layer
  size_t gsz = (size_t)3 * d.Zd * d.D;
  std::vector<double> G((size_t)std::max(d.L, 1) * gsz), Gb((size_t)std::max(d.L, 1) * d.D);
  for (int n = 0; n < d.L; ++n) {
    for (int c = 0; c < 3; ++c)
      for (int z = 0; z < d.Zd; ++z)
        for (int k = 0; k < d.D; ++k)
          G[n * gsz + ((size_t)c * d.Zd + z) * d.D + k] = hp[o.GW[n][c] + (int64_t)z * d.D + k];
    for (int k = 0; k < d.D; ++k)
      Gb[(size_t)n * d.D + k] = hp[o.Gb[n][0] + k] + hp[o.Gb[n][1] + k] + hp[o.Gb[n][2] + k];
  }
  PN_CUDA(cudaMemcpy(s->Gcat64, G.data(), G.size() * 8, cudaMemcpyHostToDevice));
  PN_CUDA(cudaMemcpy(s->Gb64, Gb.data(), Gb.size() * 8, cudaMemcpyHostToDevice));
  {
    std::vector<double> gx(d.D);
    for (int k = 0; k < d.D; ++k) gx[k] = (d.L > 0 ? Gb[k] : 0.0) + hp[o.x0 + k];
    std::vector<float> gx32(gx.begin(), gx.end());
    PN_CUDA(cudaMemcpy(s->Gbx0_64, gx.data(), gx.size() * 8, cudaMemcpyHostToDevice));
    PN_CUDA(cudaMemcpy(s->Gbx0_32, gx32.data(), gx32.size() * 4, cudaMemcpyHostToDevice));
  }
  std::vector<float> G32(G.begin(), G.end()), Gb32(Gb.begin(), Gb.end());
  PN_CUDA(cudaMemcpy(s->Gcat32, G32.data(), G32.size() * 4, cudaMemcpyHostToDevice));
  PN_CUDA(cudaMemcpy(s->Gb32, Gb32.data(), Gb32.size() * 4, cudaMemcpyHostToDevice));
  // packed sampler weights (same block order in both precisions)
  std::vector<std::pair<const double*, size_t>> blocks;
  for (int n = 0; n < d.L; ++n) {
    blocks.push_back({hp + o.hW[n], (size_t)d.D * d.Zd});
    for (int c = 0; c < 3; ++c) {
      blocks.push_back({hp + o.W1[n][c], (size_t)d.K * d.Hw});
      blocks.push_back({hp + o.W2[n][c], (size_t)d.Hw * d.Zd});
    }
    blocks.push_back({G.data() + n * gsz, gsz});
  }
  const size_t outs[6] = {(size_t)d.D, (size_t)d.D, (size_t)d.n_orb, (size_t)d.D, (size_t)d.D, 1};
  const int64_t srcs[6] = {o.kW[0], o.kW[1], o.kW[2], o.eW[0], o.eW[1], o.eW[2]};
  for (int k = 0; k < 6; ++k) blocks.push_back({hp + srcs[k], (size_t)d.D * outs[k]});
  for (int prec = 0; prec < 2; ++prec) {
    const size_t el = prec == 0 ? 8 : 4, align = 16 / el;
    StageTab& t = prec == 0 ? s->stab64 : s->stab32;
    t.n = (int)blocks.size();
    t.max_bytes = 0;
    size_t tot = 0;
    for (int b = 0; b < t.n; ++b) {
      const size_t padded = (blocks[b].second + align - 1) / align * align;
      t.off[b] = (int64_t)tot;
      t.bytes[b] = (int)(padded * el);
      t.max_bytes = std::max(t.max_bytes, t.bytes[b]);
      tot += padded;
    }
    if (prec == 0) {
      std::vector<double> pk(tot, 0.0);
      for (int b = 0; b < t.n; ++b) std::copy(blocks[b].first, blocks[b].first + blocks[b].second, pk.begin() + t.off[b]);
      PN_CUDA(cudaMemcpy(s->wpack64, pk.data(), tot * 8, cudaMemcpyHostToDevice));
    } else {
      std::vector<float> pk(tot, 0.0f);
      for (int b = 0; b < t.n; ++b) std::copy(blocks[b].first, blocks[b].first + blocks[b].second, pk.begin() + t.off[b]);
      PN_CUDA(cudaMemcpy(s->wpack32, pk.data(), tot * 4, cudaMemcpyHostToDevice));
    }
  }
  // tensor-core sampler blocks (only for shapes its tiles take)
  if (s->tcpack) {
    TcStages& t = s->tcst;
    t.n = 0;
    t.max_bytes = 0;
    std::vector<unsigned short> pk;
    // one block: W[k][n] (row stride ldw, K x Nout) -> three bf16 pieces of
    // W^T in the canonical layout (rows n padded to 16, K columns)
    auto add = [&](const double* W, int K, int Nout, int ldw) {
      const int Np = (Nout + 15) / 16 * 16;
      const size_t piece = (size_t)Np * K;
      const size_t base = pk.size();
      pk.resize(base + 3 * piece, 0);
      const size_t sbo = (size_t)K / 8 * 64;  // elements between 8-row groups
      for (int n = 0; n < Nout; ++n)
        for (int k = 0; k < K; ++k) {
          float a = (float)W[(size_t)k * ldw + n];
          unsigned short pc[3];
          for (int q = 0; q < 3; ++q) {
            uint32_t bits;
            memcpy(&bits, &a, 4);
            // round to nearest even bf16
            const uint32_t lsb = (bits >> 16) & 1u;
            bits += 0x7FFFu + lsb;
            pc[q] = (unsigned short)(bits >> 16);
            uint32_t hb = (uint32_t)pc[q] << 16;
            float hf;
            memcpy(&hf, &hb, 4);
            a = a - hf;
          }
          const size_t off = (size_t)(n / 8) * sbo + (size_t)(k / 8) * 64 + (size_t)(n % 8) * 8 + (k % 8);
          for (int q = 0; q < 3; ++q) pk[base + q * piece + off] = pc[q];
        }
      if (t.n >= PN_MAX_TC_STAGES) return;  // cannot happen within PN_MAX_LAYERS; checked below
      t.off[t.n] = (int64_t)base;
      t.bytes[t.n] = (int)(3 * piece * 2);
      t.K[t.n] = K;
      t.Np[t.n] = Np;
      t.max_bytes = std::max(t.max_bytes, t.bytes[t.n]);
      ++t.n;
    };
    for (int n = 0; n < d.L; ++n) {
      if (n > 0) add(hp + o.hW[n], d.D, d.Zd, d.Zd);  // h of layer 0 is one shared row
      for (int c = 0; c < 3; ++c) {
        if (d.ch_off[c + 1] == d.ch_off[c]) continue;
        add(hp + o.W1[n][c], d.K, d.Hw, d.Hw);
        add(hp + o.W2[n][c], d.Hw, d.Zd, d.Zd);
        add(hp + o.GW[n][c], d.Zd, d.D, d.D);
      }
    }
    add(hp + o.kW[0], d.D, d.D, d.D);
    add(hp + o.kW[1], d.D, d.D, d.D);
    add(hp + o.kW[2], d.D, d.n_orb, d.n_orb);
    add(hp + o.eW[0], d.D, d.D, d.D);
    add(hp + o.eW[1], d.D, d.D, d.D);
    add(hp + o.eW[2], d.D, 1, 1);
    int live = 0;
    for (int c = 0; c < 3; ++c) live += d.ch_off[c + 1] != d.ch_off[c];
    if (t.n != d.L * (1 + 3 * live) - 1 + 6) { pn_set_error("tensor-core stage table overflow"); return PN_EINVAL; }
    PN_CUDA(cudaMemcpy(s->tcpack, pk.data(), pk.size() * 2, cudaMemcpyHostToDevice));
    PN_CUDA(cudaMemcpy(s->tcst_dev, &t, sizeof(TcStages), cudaMemcpyHostToDevice));
  }
  return PN_OK;
}

// bf16 elements of the tensor-core sampler blocks; 0 if the shapes do not fit its tiles.
static size_t tcpack_elems(const DevSys& d) {
  if (d.D % 16 || d.Zd % 16 || d.K % 16 || d.Hw % 16 || d.D > 128) return 0;
  auto np = [](int n) { return (size_t)((n + 15) / 16 * 16); };
  size_t tot = 0;
  for (int n = 0; n < d.L; ++n) {
    tot += 3 * np(d.Zd) * d.D;
    for (int c = 0; c < 3; ++c) tot += 3 * (np(d.Hw) * d.K + np(d.Zd) * d.Hw + np(d.D) * d.Zd);
  }
  tot += 3 * d.D * (np(d.D) * 4 + np(d.n_orb) + np(1));
  return tot;
}

// Elements of the packed sampler weights (upper bound, for allocation).
static size_t wpack_elems(const DevSys& d) {
  size_t tot = 0;
  auto add = [&](size_t n) { tot += (n + 3) / 4 * 4; };
  for (int n = 0; n < d.L; ++n) {
    add((size_t)d.D * d.Zd);
    for (int c = 0; c < 3; ++c) { add((size_t)d.K * d.Hw); add((size_t)d.Hw * d.Zd); }
    add((size_t)3 * d.Zd * d.D);
  }
  add((size_t)d.D * d.D); add((size_t)d.D * d.D); add((size_t)d.D * d.n_orb);
  add((size_t)d.D * d.D); add((size_t)d.D * d.D); add((size_t)d.D);
  return tot;
}

template <>
DevNet<double> pn_devnet<double>(pn_system_s* s) {
  DevNet<double> n;
  n.p = s->p64; n.p2 = s->p2_64; n.Gcat = s->Gcat64; n.Gb = s->Gb64; n.Gbx0 = s->Gbx0_64; n.off = s->off;
  n.wpack = s->wpack64; n.stab = s->stab64;
  n.tcpack = nullptr; n.tcst = nullptr; n.tc_n = 0; n.tc_max_bytes = 0;
  return n;
}
template <>
DevNet<float> pn_devnet<float>(pn_system_s* s) {
  DevNet<float> n;
  n.p = s->p32; n.p2 = nullptr; n.Gcat = s->Gcat32; n.Gb = s->Gb32; n.Gbx0 = s->Gbx0_32; n.off = s->off;
  n.wpack = s->wpack32; n.stab = s->stab32;
  n.tcpack = s->tcpack; n.tcst = s->tcst_dev; n.tc_n = s->tcst.n; n.tc_max_bytes = s->tcst.max_bytes;
  return n;
}

// --------------------------------------------------------------- init
extern "C" int pn_init_system(const pn_system_desc* d, pn_system_t* out) {
  if (!d || !out) { pn_set_error("null argument"); return PN_EINVAL; }
  *out = nullptr;
  const int N = d->n_up + d->n_dn;
  if (d->M < 1 || d->M > PN_MAX_NUCLEI) { pn_set_error("M=%d outside 1..%d", d->M, PN_MAX_NUCLEI); return PN_EINVAL; }
  if (N < 1 || N > PN_MAX_ELECTRONS) { pn_set_error("N=%d outside 1..%d", N, PN_MAX_ELECTRONS); return PN_EINVAL; }
  if (d->n_up < 0 || d->n_dn < 0 || d->n_up > PN_MAX_SPIN || d->n_dn > PN_MAX_SPIN || d->n_up < d->n_dn) {
    pn_set_error("spin counts n_up=%d n_dn=%d invalid (need n_dn <= n_up <= %d)", d->n_up, d->n_dn, PN_MAX_SPIN);
    return PN_EINVAL;
  }
  if (d->n_orb < 1 || d->n_orb > PN_MAX_ORBITALS) { pn_set_error("n_orb=%d outside 1..%d", d->n_orb, PN_MAX_ORBITALS); return PN_EINVAL; }
  if (d->n_det < 1 || d->n_det > PN_MAX_DETS) { pn_set_error("n_det=%d outside 1..%d", d->n_det, PN_MAX_DETS); return PN_EINVAL; }
  if (d->L < 0 || d->L > PN_MAX_LAYERS) { pn_set_error("L=%d outside 0..%d", d->L, PN_MAX_LAYERS); return PN_EINVAL; }
  if (d->D < 1 || d->D > PN_MAX_DIM || d->Zd < 1 || d->Zd > PN_MAX_DIM || d->K < 1 || d->K > 64) {
    pn_set_error("network sizes D=%d Zd=%d K=%d out of range", d->D, d->Zd, d->K);
    return PN_EINVAL;
  }
  if (std::max(d->K, d->Zd) > 128) { pn_set_error("filter hidden width max(K,Zd) > 128"); return PN_EINVAL; }
  if (d->n_shells < 1 || !d->Z || !d->R || !d->shell_center || !d->shell_l || !d->shell_nprim ||
      !d->prim_exp || !d->prim_coef || !d->mo_coeffs || !d->ci || !d->params ||
      (d->n_up > 0 && !d->occ_up) || (d->n_dn > 0 && !d->occ_dn)) {
    pn_set_error("missing array in system description");
    return PN_EINVAL;
  }
  if (d->precision != PN_FP64 && d->precision != PN_MIXED) { pn_set_error("precision %d unknown", d->precision); return PN_EINVAL; }
  NetOff off = pn_net_offsets(d->D, d->Zd, d->K, d->L, d->M, d->n_orb);
  if (d->n_params != off.total) {
    pn_set_error("n_params=%lld, layout needs %lld", (long long)d->n_params, (long long)off.total);
    return PN_EINVAL;
  }
  HostSys h;
  h.M = d->M; h.N = N; h.n_up = d->n_up; h.n_dn = d->n_dn; h.n_orb = d->n_orb; h.n_det = d->n_det;
  h.n_shells = d->n_shells;
  h.Z.assign(d->Z, d->Z + d->M);
  h.R.assign(d->R, d->R + 3 * d->M);
  int nprim_tot = 0, nb = 0;
  for (int s = 0; s < d->n_shells; ++s) {
    int l = d->shell_l[s], c = d->shell_center[s], np = d->shell_nprim[s];
    if (l < -1 || l > 2 || c < 0 || c >= d->M || np < 1 || np > 16 || (l == -1 && np != 1)) {
      pn_set_error("shell %d invalid (center %d, l %d, nprim %d)", s, c, l, np);
      return PN_EINVAL;
    }
    h.sc.push_back(c); h.sl.push_back(l); h.sn.push_back(np);
    h.spo.push_back(nprim_tot); h.sbo.push_back(nb);
    nprim_tot += np;
    nb += ncart(l);
  }
  h.n_b = nb;
  h.pe.assign(d->prim_exp, d->prim_exp + nprim_tot);
  h.pc.assign(d->prim_coef, d->prim_coef + nprim_tot);
  h.mo.assign(d->mo_coeffs, d->mo_coeffs + (size_t)nb * d->n_orb);
  for (int I = 0; I < d->M; ++I)
    if (!(d->Z[I] > 0)) { pn_set_error("nuclear charge %d not positive", I); return PN_EINVAL; }
  std::vector<int> occ((size_t)d->n_det * N);
  for (int p = 0; p < d->n_det; ++p) {
    for (int k = 0; k < d->n_up; ++k) occ[(size_t)p * N + k] = d->occ_up[p * d->n_up + k];
    for (int k = 0; k < d->n_dn; ++k) occ[(size_t)p * N + d->n_up + k] = d->occ_dn[p * d->n_dn + k];
  }
  for (int v : occ)
    if (v < 0 || v >= d->n_orb) { pn_set_error("orbital index %d outside 0..%d", v, d->n_orb - 1); return PN_EINVAL; }

  // --- nuclear cusp splice coefficients (Ma et al., value at nucleus free)
  std::vector<double> crc(d->M, 0.0), cC((size_t)d->M * d->n_orb, 0.0), cS((size_t)d->M * d->n_orb, 1.0),
      cA((size_t)d->M * d->n_orb * 5, 0.0);
  std::vector<int> con((size_t)d->M * d->n_orb, 0);
  if (d->use_cusp) {
    for (int I = 0; I < d->M; ++I) {
      double rc = 0.5 / d->Z[I];
      crc[I] = rc;
      bool has_s = false;
      for (int s = 0; s < d->n_shells; ++s) has_s |= (h.sl[s] == 0 && h.sc[s] == I);
      if (!has_s) continue;
      std::vector<double> full;
      host_orbitals(h, &h.R[3 * I], full);
      for (int mu = 0; mu < d->n_orb; ++mu) {
        double gmin = 1e300, gmax = -1e300, scale = 0;
        double f0 = 0, f1, f2, fend = 0;
        for (int g = 0; g < 64; ++g) {
          double rr = rc * g / 63.0;
          double f;
          host_s_part(h, I, mu, rr, &f, &f1, &f2);
          if (g == 0) f0 = f;
          if (g == 63) fend = f;
          gmin = std::min(gmin, f);
          gmax = std::max(gmax, f);
          scale = std::max(scale, fabs(f));
        }
        if (scale < 1e-14) continue;
        double C = 0;
        if (gmin < 0 && gmax > 0) C = (fend > 0) ? gmin - 0.1 * scale : gmax + 0.1 * scale;
        double fr, fr1, fr2;
        host_s_part(h, I, mu, rc, &fr, &fr1, &fr2);
        double sg = (fr - C > 0) ? 1.0 : -1.0;
        double phi0 = d->cusp_phi0 ? d->cusp_phi0[(size_t)mu * d->M + I] : f0;
        if ((phi0 - C) * sg <= 0) {
          pn_set_error("cusp: phi0 - C has the wrong sign for orbital %d at nucleus %d", mu, I);
          return PN_EINVAL;
        }
        double eta0 = full[mu] - f0;
        double a0 = log(fabs(phi0 - C));
        double a1 = -d->Z[I] * (phi0 + eta0) / (phi0 - C);
        double X1 = log(fabs(fr - C));
        double X2 = fr1 / (fr - C);
        double X3 = fr2 / (fr - C) - X2 * X2;
        double A[3][3] = {{rc * rc, rc * rc * rc, rc * rc * rc * rc},
                          {2 * rc, 3 * rc * rc, 4 * rc * rc * rc},
                          {2.0, 6 * rc, 12 * rc * rc}};
        double b[3] = {X1 - a0 - a1 * rc, X2 - a1, X3}, x[3];
        if (!solve3(A, b, x)) { pn_set_error("cusp: singular matching system"); return PN_EINVAL; }
        size_t k = (size_t)I * d->n_orb + mu;
        con[k] = 1;
        cC[k] = C;
        cS[k] = sg;
        cA[k * 5 + 0] = a0; cA[k * 5 + 1] = a1;
        cA[k * 5 + 2] = x[0]; cA[k * 5 + 3] = x[1]; cA[k * 5 + 4] = x[2];
      }
    }
  }

  pn_system_s* s = new pn_system_s();
  s->work_mem = nullptr;
  s->tape_mem = nullptr;
  s->tape_bytes = 0;
  cudaGetDevice(&s->device);
  s->off = off;
  s->precision = d->precision;
  s->no_jastrow = d->no_jastrow ? 1 : 0;
  s->no_backflow = d->no_backflow ? 1 : 0;
  s->drift_mode = 1;
  DevSys& ds = s->ds;
  ds.N = N; ds.n_up = d->n_up; ds.n_dn = d->n_dn; ds.M = d->M; ds.n_b = nb; ds.n_orb = d->n_orb;
  ds.n_det = d->n_det; ds.n_shells = d->n_shells;
  ds.D = d->D; ds.Zd = d->Zd; ds.K = d->K; ds.L = d->L; ds.Hw = std::max(d->K, d->Zd);
  ds.Pee = N * (N - 1) / 2; ds.Pen = N * d->M; ds.Ppair = ds.Pee + ds.Pen;
  ds.r_c = d->r_c; ds.use_cusp = d->use_cusp; ds.use_gamma = d->use_gamma;
  // mixed path: the tensor-core sampler where its tiles fit (else the warp kernel)
  ds.fused_sampler = d->precision == PN_MIXED ? 4 : 1;
  // mixed systems: every float32 linear map group on tcgen05 (its split
  // accumulators make it at least as accurate as CUDA-core float32)
  ds.tensor_cores = d->precision == PN_MIXED ? 7 : 0;
  double Vnn = 0;
  for (int I = 0; I < d->M; ++I)
    for (int J = I + 1; J < d->M; ++J) {
      double dx = d->R[3 * I] - d->R[3 * J], dy = d->R[3 * I + 1] - d->R[3 * J + 1], dz = d->R[3 * I + 2] - d->R[3 * J + 2];
      Vnn += d->Z[I] * d->Z[J] / sqrt(dx * dx + dy * dy + dz * dz);
    }
  ds.Vnn = Vnn;
  std::vector<double> fmu(d->K), fis(d->K);
  for (int k = 0; k < d->K; ++k) {
    double q = (double)(k + 1) / (d->K + 1);
    double sig = (1.0 + d->r_c * q) / 7.0;
    fmu[k] = d->r_c * q * q;
    fis[k] = 1.0 / (sig * sig);
  }
  int err = PN_OK;
  ds.Z = dev_upload(s, d->Z, d->M, &err);
  ds.R = dev_upload(s, d->R, 3 * d->M, &err);
  ds.sh_center = dev_upload(s, h.sc.data(), h.sc.size(), &err);
  ds.sh_l = dev_upload(s, h.sl.data(), h.sl.size(), &err);
  ds.sh_nprim = dev_upload(s, h.sn.data(), h.sn.size(), &err);
  ds.sh_poff = dev_upload(s, h.spo.data(), h.spo.size(), &err);
  ds.sh_boff = dev_upload(s, h.sbo.data(), h.sbo.size(), &err);
  ds.pexp = dev_upload(s, h.pe.data(), h.pe.size(), &err);
  ds.pcoef = dev_upload(s, h.pc.data(), h.pc.size(), &err);
  ds.mo = dev_upload(s, h.mo.data(), h.mo.size(), &err);
  ds.occ = dev_upload(s, occ.data(), occ.size(), &err);
  // excitation table relative to determinant 0 (see DevSys::xtab)
  {
    const int hdr = 2 * (1 + PN_MAX_ORBITALS);
    std::vector<int> xt(hdr + (size_t)d->n_det * 2 * PN_TAB_REC, 0);
    bool ok = true;
    size_t wstride = 0;
    for (int sg = 0; sg < 2 && ok; ++sg) {
      const int n = sg ? d->n_dn : d->n_up, e0 = sg ? d->n_up : 0;
      std::vector<int> occ0(occ.begin() + e0, occ.begin() + e0 + n), V;
      for (int p = 0; p < d->n_det; ++p)
        for (int c = 0; c < n; ++c) {
          const int mu = occ[(size_t)p * N + e0 + c];
          if (std::find(occ0.begin(), occ0.end(), mu) == occ0.end() && std::find(V.begin(), V.end(), mu) == V.end())
            V.push_back(mu);
        }
      std::sort(V.begin(), V.end());
      if (n > PN_TAB_NMAX || (int)V.size() > PN_TAB_VMAX) { ok = false; break; }
      xt[sg * (1 + PN_MAX_ORBITALS)] = (int)V.size();
      for (size_t v = 0; v < V.size(); ++v) xt[sg * (1 + PN_MAX_ORBITALS) + 1 + v] = V[v];
      auto parity = [](const std::vector<int>& a) {
        int inv = 0;
        for (size_t i = 0; i < a.size(); ++i)
          for (size_t j = i + 1; j < a.size(); ++j) inv += a[i] > a[j];
        return (inv & 1) ? -1 : 1;
      };
      int k3 = 0;
      size_t minor_doubles = 0;
      for (int p = 0; p < d->n_det && ok; ++p) {
        // positions of determinant p holding a reference orbital (U, at
        // reference position j) and holding a virtual one (C)
        std::vector<int> U, J, C, used(n, 0);
        for (int c = 0; c < n; ++c) {
          const int mu = occ[(size_t)p * N + e0 + c];
          const int j = (int)(std::find(occ0.begin(), occ0.end(), mu) - occ0.begin());
          if (j < n) {
            if (used[j]) { ok = false; break; }  // repeated orbital: leave it to the direct kernel
            used[j] = 1;
            U.push_back(c);
            J.push_back(j);
          } else {
            C.push_back(c);
          }
        }
        if (!ok) break;
        const int k = (int)C.size();
        if (k > PN_TAB_KMAX) { ok = false; break; }
        std::vector<int> H;
        for (int j = 0; j < n; ++j) if (!used[j]) H.push_back(j);
        // block-triangular order: rows (J, H), columns (U, C)
        std::vector<int> rows(J), cols(U);
        rows.insert(rows.end(), H.begin(), H.end());
        cols.insert(cols.end(), C.begin(), C.end());
        int* rec = &xt[hdr + ((size_t)2 * p + sg) * PN_TAB_REC];
        rec[0] = k;
        rec[1] = parity(rows) * parity(cols);
        for (int q = 0; q < k; ++q) {
          rec[2 + q] = H[q];
          const int mu = occ[(size_t)p * N + e0 + C[q]];
          rec[2 + PN_TAB_KMAX + q] = (int)(std::find(V.begin(), V.end(), mu) - V.begin());
        }
        k3 += k * k * k;
        minor_doubles += (size_t)k * k + 3;
      }
      const size_t nv = V.size(), ncol = n + nv, n3 = 3 * (size_t)N;
      // the packed minors reuse the dead matrices A..B where they fit
      const size_t dead = 3 * n * ncol + 3 * (size_t)n * n;
      wstride = std::max(wstride, 3 * n * ncol + 3 * (size_t)n * n + 4 * n * nv + n3 + n3 * n * nv + n + 2 +
                                      (minor_doubles <= dead ? 0 : minor_doubles));
      ds.tab_nv[sg] = (int)nv;
      ds.tab_k3[sg] = k3;
    }
    ds.xtab = nullptr;
    ds.tab_wstride = 0;
    if (ok) {
      ds.xtab = dev_upload(s, xt.data(), xt.size(), &err);
      ds.tab_wstride = (int)((wstride + 1) & ~(size_t)1);
    }
  }
  ds.ci = dev_upload(s, d->ci, d->n_det, &err);
  ds.cusp_rc = dev_upload(s, crc.data(), crc.size(), &err);
  ds.cusp_on = dev_upload(s, con.data(), con.size(), &err);
  ds.cusp_C = dev_upload(s, cC.data(), cC.size(), &err);
  ds.cusp_s = dev_upload(s, cS.data(), cS.size(), &err);
  ds.cusp_a = dev_upload(s, cA.data(), cA.size(), &err);
  {
    // pairs grouped by filter channel: same spin, opposite spin, nucleus
    std::vector<int> chp;
    for (int c = 0; c < 3; ++c) {
      ds.ch_off[c] = (int)chp.size();
      for (int a = 0; a < N; ++a)
        for (int b = a + 1; b < N; ++b) {
          const int ch = ((a < d->n_up) == (b < d->n_up)) ? 0 : 1;
          if (ch == c) chp.push_back(pn_pair_index(a, b, N));
        }
      if (c == 2)
        for (int q = 0; q < N * d->M; ++q) chp.push_back(ds.Pee + q);
    }
    ds.ch_off[3] = (int)chp.size();
    ds.ch_pairs = dev_upload(s, chp.data(), chp.size(), &err);
    std::vector<int> pos(chp.size());
    for (int c = 0; c < 3; ++c)
      for (int q = ds.ch_off[c]; q < ds.ch_off[c + 1]; ++q) pos[chp[q]] = q - ds.ch_off[c];
    ds.ch_pos = dev_upload(s, pos.data(), pos.size(), &err);
  }
  {
    // nucleus per electron for walker initialisation: the nuclei repeated
    // Z_I times; up electron k takes entry 2k, down electron k entry 2k + 1
    std::vector<int> lst, nuc(N);
    for (int I = 0; I < d->M; ++I)
      for (int k = 0; k < (int)llround(d->Z[I]); ++k) lst.push_back(I);
    if (lst.empty()) lst.push_back(0);
    for (int k = 0; k < d->n_up; ++k) nuc[k] = lst[(2 * k) % lst.size()];
    for (int k = 0; k < d->n_dn; ++k) nuc[d->n_up + k] = lst[(2 * k + 1) % lst.size()];
    ds.nuc = dev_upload(s, nuc.data(), nuc.size(), &err);
  }
  {
    int zero = 0;
    ds.dev_err = dev_upload(s, &zero, 1, &err);
  }
  ds.feat_mu = dev_upload(s, fmu.data(), fmu.size(), &err);
  ds.feat_isig2 = dev_upload(s, fis.data(), fis.size(), &err);
  {
    auto f32 = [&](const double* src, size_t n) {
      std::vector<float> v(src, src + n);
      return dev_upload(s, v.data(), v.size(), &err);
    };
    ds.R32 = f32(d->R, 3 * (size_t)d->M);
    ds.pexp32 = f32(h.pe.data(), h.pe.size());
    ds.pcoef32 = f32(h.pc.data(), h.pc.size());
    ds.mo32 = f32(h.mo.data(), h.mo.size());
    ds.cusp_rc32 = f32(crc.data(), crc.size());
    ds.cusp_C32 = f32(cC.data(), cC.size());
    ds.cusp_s32 = f32(cS.data(), cS.size());
    ds.cusp_a32 = f32(cA.data(), cA.size());
  }
  {
    std::vector<float> fmu32(fmu.begin(), fmu.end()), fis32(fis.begin(), fis.end());
    ds.feat_mu32 = dev_upload(s, fmu32.data(), fmu32.size(), &err);
    ds.feat_isig2_32 = dev_upload(s, fis32.data(), fis32.size(), &err);
  }
  s->p64 = dev_upload<double>(s, nullptr, off.total, &err);
  s->p32 = dev_upload<float>(s, nullptr, off.total, &err);
  s->p2_64 = dev_upload<float>(s, nullptr, 2 * (size_t)off.total, &err);
  size_t gsz = (size_t)std::max(d->L, 1) * 3 * d->Zd * d->D;
  s->Gcat64 = dev_upload<double>(s, nullptr, gsz, &err);
  s->Gb64 = dev_upload<double>(s, nullptr, (size_t)std::max(d->L, 1) * d->D, &err);
  s->Gcat32 = dev_upload<float>(s, nullptr, gsz, &err);
  s->Gbx0_64 = dev_upload<double>(s, nullptr, (size_t)d->D, &err);
  s->Gbx0_32 = dev_upload<float>(s, nullptr, (size_t)d->D, &err);
  s->Gb32 = dev_upload<float>(s, nullptr, (size_t)std::max(d->L, 1) * d->D, &err);
  s->wpack64 = dev_upload<double>(s, nullptr, wpack_elems(ds), &err);
  s->wpack32 = dev_upload<float>(s, nullptr, wpack_elems(ds), &err);
  s->tcst.n = 0;
  s->tcpack = nullptr;
  s->tcst_dev = nullptr;
  if (size_t te = tcpack_elems(ds)) {
    s->tcpack = dev_upload<unsigned short>(s, nullptr, te, &err);
    s->tcst_dev = (TcStages*)dev_upload<unsigned char>(s, nullptr, sizeof(TcStages), &err);
  }
  if (err != PN_OK) {
    pn_set_error("device allocation/upload failed during init");
    free_all(s);
    delete s;
    return err;
  }
  if (int e = upload_params(s, d->params)) { free_all(s); delete s; return e; }
  // workspace
  s->Wc = std::max(1, d->max_walkers);
  s->Tjet = 3 * N + 2;
  int elem = d->precision == PN_FP64 ? 8 : 4;
  s->work_bytes = pn_work_bytes(ds, s->Wc, s->Tjet, elem);
  if (cudaMalloc(&s->work_mem, s->work_bytes) != cudaSuccess) {
    cudaGetLastError();
    pn_set_error("workspace of %zu bytes for %d walkers does not fit", s->work_bytes, s->Wc);
    s->work_mem = nullptr;
    free_all(s);
    delete s;
    return PN_ENOMEM;
  }
  char* end;
  if (d->precision == PN_FP64) {
    s->w64 = pn_carve_work<double>(ds, s->Wc, s->Tjet, s->work_mem);
    end = s->w64.end;
  } else {
    s->w32 = pn_carve_work<float>(ds, s->Wc, s->Tjet, s->work_mem);
    end = s->w32.end;
  }
  if (end > (char*)s->work_mem + s->work_bytes) {
    pn_set_error("workspace layout exceeds its allocation");
    free_all(s);
    delete s;
    return PN_EINVAL;
  }
  // mixed handles: the local-energy guard, on by default (jets perturbed at
  // the relative and the term scale, tau = 5e-5 Ha)
  if (d->precision == PN_MIXED) {
    const int cap = std::min(s->Wc, 1024);
    const size_t gb = pn_guard_bytes(ds, s->Wc, cap);
    if (cudaMalloc(&s->guard_mem, gb) != cudaSuccess) {
      cudaGetLastError();
      pn_set_error("local-energy guard of %zu bytes does not fit", gb);
      s->guard_mem = nullptr;
      free_all(s);
      delete s;
      return PN_ENOMEM;
    }
    s->guard = pn_carve_guard(ds, s->Wc, cap, s->guard_mem);
    s->guard.net64 = pn_devnet<double>(s);
    s->guard.tau = 5e-5;
    s->ds.guard_probe = 2;
    PN_CUDA(cudaMemset(s->guard.n_total, 0, 8));
  }
  *out = s;
  return PN_OK;
}

extern "C" int pn_destroy_system(pn_system_t s) {
  if (!s) return PN_OK;
  free_all(s);
  delete s;
  return PN_OK;
}

extern "C" int pn_set_params(pn_system_t s, const double* params, int64_t n) {
  if (!s || !params) { pn_set_error("null argument"); return PN_EINVAL; }
  if (n != s->off.total) { pn_set_error("n_params=%lld, expected %lld", (long long)n, (long long)s->off.total); return PN_EINVAL; }
  std::vector<double> hp(n);
  if (pn_is_device_ptr(params)) {
    PN_CUDA(cudaMemcpy(hp.data(), params, n * 8, cudaMemcpyDeviceToHost));
  } else {
    memcpy(hp.data(), params, n * 8);
  }
  PN_CUDA(cudaDeviceSynchronize());
  return upload_params(s, hp.data());
}

extern "C" int64_t pn_num_params(pn_system_t s) { return s ? s->off.total : -1; }
extern "C" size_t pn_workspace_bytes(pn_system_t s) { return s ? s->work_bytes : 0; }
