// AdamW parameter update for VMC training (Methods, ansatz optimisation:
// Adam with decoupled weight decay after Loshchilov and Hutter, the total
// energy being the loss).  One thread per parameter, float64 throughout.
//
//   m <- b1 m + (1 - b1) g,   v <- b2 v + (1 - b2) g^2,
//   m^ = m / (1 - b1^t),      v^ = v / (1 - b2^t),
//   theta <- theta - lr (m^ / (sqrt(v^) + eps) + wd theta)
//
// (the weight decay is applied to the parameter, decoupled from the
// gradient moments).
#include <math.h>

#include "pn_internal.cuh"

namespace {

__global__ void k_adamw(double* __restrict__ theta, const double* __restrict__ g, double* __restrict__ m,
                        double* __restrict__ v, int64_t n, double lr, double b1, double b2, double eps, double wd,
                        double c1, double c2) {
  const int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double gi = g[i];
  const double mi = b1 * m[i] + (1.0 - b1) * gi;
  const double vi = b2 * v[i] + (1.0 - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const double mh = mi / c1, vh = vi / c2;
  theta[i] = theta[i] - lr * (mh / (sqrt(vh) + eps) + wd * theta[i]);
}

}  // namespace

extern "C" int pn_adamw_step(double* theta, const double* grad, double* m, double* v, int64_t n, double lr,
                             double beta1, double beta2, double eps, double weight_decay, int64_t t, void* stream) {
  if (n < 0 || (n > 0 && (!theta || !grad || !m || !v)) || t < 1 || !(beta1 >= 0 && beta1 < 1) ||
      !(beta2 >= 0 && beta2 < 1) || !(eps > 0) || !(lr >= 0) || !(weight_decay >= 0)) {
    pn_set_error("pn_adamw_step: bad arguments");
    return PN_EINVAL;
  }
  if (n == 0) return PN_OK;
  if (!pn_is_device_ptr(theta) || !pn_is_device_ptr(grad) || !pn_is_device_ptr(m) || !pn_is_device_ptr(v)) {
    pn_set_error("pn_adamw_step takes device buffers");
    return PN_EINVAL;
  }
  const double c1 = 1.0 - pow(beta1, (double)t), c2 = 1.0 - pow(beta2, (double)t);
  cudaStream_t st = (cudaStream_t)stream;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  PN_LAUNCH("k_adamw", st, k_adamw<<<blocks, 256, 0, st>>>(theta, grad, m, v, n, lr, beta1, beta2, eps, weight_decay, c1, c2));
  return PN_OK;
}
