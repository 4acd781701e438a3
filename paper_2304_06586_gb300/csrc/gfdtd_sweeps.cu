// gfdtd_sweeps.cu -- batched parameter sweeps on the GPU: the von Neumann
// stability map of the generalized scheme (Sec. 5, App. A) and the star
// transfer-matrix scattering of moving layered stacks (App. B.3).  Both are
// FP64 throughout: the stability decision sits at |zeta| = 1 and the
// transfer matrices multiply phases over many layers.
#include "../../include/gfdtd.h"

#include <cuda_runtime.h>

#include <cstdint>

namespace {

struct cd {
  double re, im;
};
__device__ __forceinline__ cd mk(double re, double im) { return cd{re, im}; }
__device__ __forceinline__ cd operator+(cd a, cd b) { return mk(a.re + b.re, a.im + b.im); }
__device__ __forceinline__ cd operator-(cd a, cd b) { return mk(a.re - b.re, a.im - b.im); }
__device__ __forceinline__ cd operator*(cd a, cd b) {
  return mk(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
__device__ __forceinline__ cd operator*(double s, cd a) { return mk(s * a.re, s * a.im); }
__device__ __forceinline__ cd cdiv(cd a, cd b) {
  // a / b with the larger component of b factored out (Smith's method)
  if (fabs(b.re) >= fabs(b.im)) {
    const double r = b.im / b.re, d = b.re + b.im * r;
    return mk((a.re + a.im * r) / d, (a.im - a.re * r) / d);
  }
  const double r = b.re / b.im, d = b.re * r + b.im;
  return mk((a.re * r + a.im) / d, (a.im * r - a.re) / d);
}
// principal square root: with m = |z|, sqrt(z) = u + i v, u = sqrt((m + x) / 2)
// for x >= 0 (v = y / 2u); for x < 0 take v first to avoid cancellation
__device__ __forceinline__ cd csqrt(cd z) {
  const double m = hypot(z.re, z.im);
  if (m == 0.0) return mk(0.0, 0.0);
  if (z.re >= 0.0) {
    const double u = sqrt(0.5 * (m + z.re));
    return mk(u, z.im / (2.0 * u));
  }
  const double v = copysign(sqrt(0.5 * (m - z.re)), z.im);
  return mk(z.im / (2.0 * v), v);
}
__device__ __forceinline__ double cabs(cd z) { return hypot(z.re, z.im); }
__device__ __forceinline__ cd cexpi(double phi) {   // exp(i phi)
  double s, c;
  sincos(phi, &s, &c);
  return mk(c, s);
}

// ------------------------------------------------------------------ stability map
//
// Plane wave B, D ~ xi^k zeta^n, xi = exp(i theta) (Eq. PW_test_field): one
// step of Sec. 4 with the Table 1 stencils maps (B, D) to G (B, D), with
//   E* = ie D - bc (bsum / 2) B,            B' = (1 - beta S adv) B - S curl E*
//   H* = im B' - bc cos(theta / 2) D,      D' = (1 - beta S adv) D - S curl H*
// curl = 2 i sin(theta / 2) (the half-cell difference), and for v >= 0 (columns
// Ba, dBa) bsum = e^{-i theta/2} + e^{-3i theta/2}, adv = 1 - e^{-i theta}; for
// v < 0 (Bb, dBb) the mirror images.  Moving perturbation: ie = 1/eps,
// im = 1/mu, bc = beta; moving matter: the solved star relations (Eq.
// const_3d).  The result is the largest eigenvalue modulus of G over the
// samples theta_j = pi (j + 1) / n_theta.

// h = e^{+i theta / 2} of the sample.
__device__ double max_zeta_at(double S, double beta, double ie, double im, double bc, cd h) {
  const cd w = h * h;                                // e^{+i theta}
  const cd h3 = h * w;                               // e^{+3i theta/2}
  cd bsum, adv;
  if (beta >= 0.0) {
    bsum = mk(h.re, -h.im) + mk(h3.re, -h3.im);
    adv = mk(1.0 - w.re, w.im);
  } else {
    bsum = h3 + h;
    adv = mk(w.re - 1.0, w.im);
  }
  const cd curl = mk(0.0, 2.0 * h.im);
  const double avg = h.re;
  const cd diag = mk(1.0, 0.0) - (beta * S) * adv;
  const cd EsB = (-0.5 * bc) * bsum;
  const cd BB = diag - S * (curl * EsB);
  const cd BD = (-S * ie) * curl;
  const cd HB = im * BB;
  const cd HD = im * BD - mk(bc * avg, 0.0);
  const cd DB = (-S) * (curl * HB);
  const cd DD = diag - S * (curl * HD);
  const cd half_tr = 0.5 * (BB + DD);
  const cd det = BB * DD - BD * DB;
  const cd r = csqrt(half_tr * half_tr - det);
  const double a = cabs(half_tr + r), b = cabs(half_tr - r);
  return a > b ? a : b;
}

__global__ void stability_map_kernel(int64_t n, const double* __restrict__ S, const double* __restrict__ beta,
                                     const double* __restrict__ eps, const double* __restrict__ mu,
                                     const int* __restrict__ kind, int n_theta, double* __restrict__ out) {
  const int lane = threadIdx.x & 31;
  const int64_t warps = (int64_t)gridDim.x * (blockDim.x >> 5);
  for (int64_t i = (int64_t)blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5); i < n; i += warps) {
    const double s = S[i], b = beta[i], e = eps[i], m = mu[i];
    double ie, im, bc;
    if (kind[i] == GFDTD_PERTURBATION) {
      ie = 1.0 / e;
      im = 1.0 / m;
      bc = b;
    } else {   // E* = D / eps_m - beta_c B, H* = B / mu_m - beta_c D
      const double den = e * m - b * b, g = 1.0 - b * b;
      ie = g * m / den;
      im = g * e / den;
      bc = b * g / den;
    }
    // e^{i theta_j / 2} advances by e^{i 16 pi / n_theta} from one sample of the
    // lane to the next; it is recomputed from the angle every 16 samples, which
    // keeps the accumulated rounding near 1e-15.
    const double half_step = 3.14159265358979323846 / (double)n_theta * 0.5;   // theta / 2 per j
    const cd rot = cexpi(32.0 * half_step);
    double worst = 0.0;
    cd h = mk(1.0, 0.0);
    int k = 0;
    for (int j = lane; j < n_theta; j += 32, ++k) {
      if ((k & 15) == 0) h = cexpi((double)(j + 1) * half_step);
      else h = h * rot;
      worst = fmax(worst, max_zeta_at(s, b, ie, im, bc, h));
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) worst = fmax(worst, __shfl_xor_sync(0xffffffffu, worst, o));
    if (lane == 0) out[i] = worst;
  }
}

// ------------------------------------------------------------------ star transfer matrix
//
// App. B.3 for a stack moving at beta: in the frame of the structure every
// wave has the frequency Omega = omega (1 - n_0 beta), the +z and -z waves of
// layer m have lab wavenumbers n Omega / (1 -+ n beta), and the star
// amplitudes u+ = E+ (1 - n beta), u- = E- (1 + n beta) are continuous through
// each interface in the way E* = u+ + u- and H* = (u+ - u-) / eta (Eq. cont,
// Eq. star) require.  The chain of interface and propagation matrices maps
// (u+, u-) of the first medium to the last; no wave enters from the right.

__global__ void star_tmm_kernel(int64_t n_stacks, const int64_t* __restrict__ off,
                                const double* __restrict__ eps, const double* __restrict__ mu,
                                const double* __restrict__ thick, const double* __restrict__ beta,
                                int64_t n_freq, const double* __restrict__ omega, double* __restrict__ T,
                                double* __restrict__ G) {
  const int64_t total = n_stacks * n_freq;
  for (int64_t q = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; q < total;
       q += (int64_t)gridDim.x * blockDim.x) {
    const int64_t s = q / n_freq, f = q - s * n_freq;
    const int64_t l0 = off[s], nl = off[s + 1] - l0;
    if (nl < 2) {   // no interface: not a stack
      T[2 * q] = T[2 * q + 1] = G[2 * q] = G[2 * q + 1] = nan("");
      continue;
    }
    const double b = beta[s], w = omega[f];
    const double n0 = sqrt(eps[l0] * mu[l0]);
    const double Om = w * (1.0 - n0 * b);
    cd M00 = mk(1.0, 0.0), M01 = mk(0.0, 0.0), M10 = mk(0.0, 0.0), M11 = mk(1.0, 0.0);
    double eta_a = sqrt(mu[l0] / eps[l0]);
    for (int64_t m = 0; m + 1 < nl; ++m) {
      const double em = eps[l0 + m + 1], mm = mu[l0 + m + 1];
      const double eta_b = sqrt(mm / em);
      const double p = 0.5 * (1.0 + eta_b / eta_a), r = 0.5 * (1.0 - eta_b / eta_a);
      // interface: [[p, r], [r, p]] M
      const cd a00 = p * M00 + r * M10, a01 = p * M01 + r * M11;
      const cd a10 = r * M00 + p * M10, a11 = r * M01 + p * M11;
      M00 = a00; M01 = a01; M10 = a10; M11 = a11;
      if (m + 2 < nl) {   // propagation through layer m + 1
        const double nn = sqrt(em * mm), L = thick[l0 + m + 1];
        const cd ep = cexpi(nn * Om / (1.0 - nn * b) * L);
        const cd em_ = cexpi(-nn * Om / (1.0 + nn * b) * L);
        M00 = ep * M00; M01 = ep * M01;
        M10 = em_ * M10; M11 = em_ * M11;
      }
      eta_a = eta_b;
    }
    const double nN = sqrt(eps[l0 + nl - 1] * mu[l0 + nl - 1]);
    const cd u1p = mk(1.0 - n0 * b, 0.0);
    const cd u1m = cdiv(mk(0.0, 0.0) - M10 * u1p, M11);
    const cd uNp = M00 * u1p + M01 * u1m;
    const cd t = (1.0 / (1.0 - nN * b)) * uNp, g = (1.0 / (1.0 + n0 * b)) * u1m;
    T[2 * q] = t.re;
    T[2 * q + 1] = t.im;
    G[2 * q] = g.re;
    G[2 * q + 1] = g.im;
  }
}

int sm_count() {
  static int n = 0;
  if (n == 0) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || n <= 0)
      n = 1;
  }
  return n;
}

}  // namespace

extern "C" gfdtd_status gfdtd_stability_map(int64_t n, const double* S, const double* beta, const double* eps_r,
                                            const double* mu_r, const int* kind, int n_theta, double* out,
                                            void* cuda_stream) {
  if (n < 0 || n_theta < 1) return GFDTD_E_ARG;
  if (n == 0) return GFDTD_OK;
  if (!S || !beta || !eps_r || !mu_r || !kind || !out) return GFDTD_E_ARG;
  const int64_t want = (n + 7) / 8;   // blocks of 8 warps, one point per warp
  const int grid = (int)(want < 64LL * sm_count() ? want : 64LL * sm_count());
  stability_map_kernel<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(n, S, beta, eps_r, mu_r, kind, n_theta, out);
  return cudaGetLastError() == cudaSuccess ? GFDTD_OK : GFDTD_E_CUDA;
}

extern "C" gfdtd_status gfdtd_star_tmm(int64_t n_stacks, const int64_t* layer_off, const double* eps_r,
                                       const double* mu_r, const double* thick, const double* beta,
                                       int64_t n_freq, const double* omega, double* T, double* Gamma,
                                       void* cuda_stream) {
  if (n_stacks < 0 || n_freq < 0) return GFDTD_E_ARG;
  if (n_stacks == 0 || n_freq == 0) return GFDTD_OK;
  if (!layer_off || !eps_r || !mu_r || !thick || !beta || !omega || !T || !Gamma) return GFDTD_E_ARG;
  const int64_t total = n_stacks * n_freq;
  const int64_t want = (total + 255) / 256;
  const int grid = (int)(want < 32LL * sm_count() ? want : 32LL * sm_count());
  star_tmm_kernel<<<grid, 256, 0, (cudaStream_t)cuda_stream>>>(n_stacks, layer_off, eps_r, mu_r, thick, beta,
                                                                n_freq, omega, T, Gamma);
  return cudaGetLastError() == cudaSuccess ? GFDTD_OK : GFDTD_E_CUDA;
}
