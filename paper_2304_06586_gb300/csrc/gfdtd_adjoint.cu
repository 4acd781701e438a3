// gfdtd_adjoint.cu -- reverse-time discrete adjoint of the batched step.
//
// For moving perturbation the step n maps (B^{n-1}, D^{n-1/2}) linearly to
// (B^n, D^{n+1/2}) (Sec. 4 with Table 1; the source adds a constant):
//   E'_k = se_k D_k - cb Bsum_k,   B'_j = a B_j + c B_up(j) + E'_j - E'_{j+1},
//   H'_j = sm_j B'_j - cb (D_j + D_{j+1}),   D'_k = a D_k + c D_up(k) + H'_{k-1} - H'_k,
// with E' = S E*, H' = S H*.  adjoint_step applies the transpose, gathered per
// cell, to the adjoint fields (lB', lD') of (B^n, D^{n+1/2}):
//   lH_j  = lD'_{j+1} - lD'_j,          lBt_j = lB'_j + sm_j lH_j,
//   lE_k  = lBt_k - lBt_{k-1},
//   lD_k  = a lD'_k + c lD'_dn(k) - cb (lH_k + lH_{k-1}) + se_k lE_k,
//   lB_j  = a lBt_j + c lBt_dn(j) - cb (lE_{j+1} + lE_{j+2})   (v >= 0)
//                                 - cb (lE_j + lE_{j-1})       (v <  0),
// where dn is the downwind neighbour (the cell whose upwind neighbour is k)
// and every quantity outside [0, nz) is zero (the forward ghosts).  The
// permittivity enters through se = S/eps at level n-1/2:
//   dL/deps_k += lE_k * (-S D_k^{n-1/2} / eps_k^2) = lE_k * (-se_k^2 D_k / S),
// scattered onto the profile values with the interpolation weights.
#include "gfdtd_block.cuh"

namespace gfdtd {



// Weights of eps at moving coordinate xi on the profile values: (i0, w0), (i1, w1).
__device__ __forceinline__ void eps_weights(const InstDev& I, const long long* zq, long long xi,
                                            int& i0, double& w0, int& i1, double& w1) {
  if (!(I.flags & F_LINEAR)) {
    int lo = 0, hi = I.n - 1;                 // count of boundaries <= xi
    while (lo < hi) { const int mid = (lo + hi) >> 1; if (__ldg(zq + mid) <= xi) lo = mid + 1; else hi = mid; }
    i0 = lo; w0 = 1.0; i1 = lo; w1 = 0.0;
    return;
  }
  const int n = I.n;
  if (xi <= __ldg(zq)) { i0 = i1 = 0; w0 = 1.0; w1 = 0.0; return; }
  if (xi >= __ldg(zq + n - 1)) { i0 = i1 = n - 1; w0 = 1.0; w1 = 0.0; return; }
  int lo = 0, hi = n;                         // last knot <= xi
  while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (__ldg(zq + mid) <= xi) lo = mid; else hi = mid; }
  const double w = (double)(xi - __ldg(zq + lo)) / (double)(__ldg(zq + lo + 1) - __ldg(zq + lo));
  i0 = lo; w0 = 1.0 - w; i1 = lo + 1; w1 = w;
}

// Sum v over the lanes of the warp that share `key` (keys are non-decreasing
// across lanes) and add the sum once, from the segment's first lane.
__device__ __forceinline__ void segmented_atomic_add(double* base, int key, double v, bool active) {
  const int lane = threadIdx.x & 31;
  if (!active) key = -1 - lane;               // inactive lanes form singleton segments
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_down_sync(FULL, v, o);
    const int tk = __shfl_down_sync(FULL, key, o);
    if (lane + o < 32 && tk == key) v += t;
  }
  const int prev = __shfl_up_sync(FULL, key, 1);
  if (active && (lane == 0 || prev != key) && v != 0.0) atomicAdd(base + key, v);
}

__global__ void __launch_bounds__(256) adjoint_step_kernel(const AdjArgs A) {
  const int2 tl = A.tiles[blockIdx.x];
  const InstDev I = A.inst[tl.x];
  const int k = tl.y + threadIdx.x;
  const int nz = I.nz;
  const bool valid = k < nz;
  const float* lBn = A.lBn + I.off;
  const float* lDn = A.lDn + I.off;
  auto lb = [&](int j) -> double { return (j >= 0 && j < nz) ? (double)lBn[j] : 0.0; };
  auto ld = [&](int j) -> double { return (j >= 0 && j < nz) ? (double)lDn[j] : 0.0; };
  const bool pos = (I.flags & F_POS) != 0;
  const double a = I.a, c = I.c, cb = I.cb, S = I.S;
  const long long n = A.n;
  const long long offH = I.dq * (2 * n) - HALF_CELL;
  const bool mu_const = (I.flags & F_MU_CONST) != 0;
  const double sm0 = __ldg(A.tb.tabH + I.tab).x;
  auto sm = [&](int j) -> double {
    if (mu_const) return sm0;
    double x, y;
    node_coef<false, false>(I, A.tb, offH, j, x, y);
    return x;
  };
  auto lH = [&](int j) -> double { return (j >= 0 && j < nz) ? ld(j + 1) - ld(j) : 0.0; };
  auto lBt = [&](int j) -> double { return (j >= 0 && j < nz) ? lb(j) + sm(j) * lH(j) : 0.0; };
  auto lE = [&](int j) -> double { return (j >= 0 && j < nz) ? lBt(j) - lBt(j - 1) : 0.0; };

  int gkey0 = 0, gkey1 = 0;
  double gval0 = 0.0, gval1 = 0.0;
  if (valid) {
    const long long offE = I.dq * (2 * n - 1);
    double se, cbx;
    node_coef<false, true>(I, A.tb, offE, k, se, cbx);
    const double lEk = lE(k);
    const double lDk = a * ld(k) + c * ld(pos ? k + 1 : k - 1) - cb * (lH(k) + lH(k - 1)) + se * lEk;
    const double lBk = a * lBt(k) + c * lBt(pos ? k + 1 : k - 1)
                     - cb * (pos ? lE(k + 1) + lE(k + 2) : lE(k) + lE(k - 1));
    A.lD[I.off + k] = (float)lDk;
    A.lB[I.off + k] = (float)lBk;
    const double gE = lEk * (-se * se * (double)A.Dold[I.off + k] / S);
    double w0, w1;
    eps_weights(I, A.tb.zq + I.tab, ((long long)k << 32) - offE, gkey0, w0, gkey1, w1);
    gval0 = gE * w0;
    gval1 = gE * w1;
  }
  double* g = A.grad + I.tab;
  segmented_atomic_add(g, gkey0, gval0, valid);
  segmented_atomic_add(g, gkey1, gval1, valid && (I.flags & F_LINEAR));
}

// The probe term of step n: F_n = D^{n+1/2}_p se_p / S = D_p / eps_p (level
// n+1/2) with dL/dF_n = g[inst]; adds g se_p / S to lD at the probe node and
// g dF/deps = g (-D_p / eps_p^2) to dL/deps.  One thread per instance.


__global__ void probe_adjoint_kernel(const ProbeAdjArgs A) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= A.n_inst) return;
  const InstDev I = A.inst[i];
  const int kp = A.probe_node[i];
  const double g = A.gn[i];
  if (kp < 0 || g == 0.0) return;
  const long long off = I.dq * (2 * A.n + 1);
  double se, cb;
  node_coef<false, true>(I, A.tb, off, kp, se, cb);
  A.lD[I.off + kp] += (float)(g * se / I.S);
  // F = D / eps: dF/deps = -D / eps^2 = -D se^2 / S^2
  const double gE = g * (-(double)A.Dnew[I.off + kp] * se * se / (I.S * I.S));
  int i0, i1;
  double w0, w1;
  eps_weights(I, A.tb.zq + I.tab, ((long long)kp << 32) - off, i0, w0, i1, w1);
  atomicAdd(A.grad + I.tab + i0, gE * w0);
  if (I.flags & F_LINEAR) atomicAdd(A.grad + I.tab + i1, gE * w1);
}

// dL/dF_n per instance for one segment: 2 S sum_f (Re X_f cos(w t) + Im X_f sin(w t)).


__global__ void loss_source_kernel(const SourceAdjArgs A) {
  const int idx = blockIdx.x * blockDim.x + threadIdx.x;
  if (idx >= A.n_inst * A.steps) return;
  const int i = idx % A.n_inst, s = idx / A.n_inst;
  const long long n = A.n_first + s;
  const double t = (double)(2 * n + 1) * A.S * 0.5;
  double g = 0.0;
  for (int f = 0; f < A.nb; ++f) {
    const int b = A.bin0[i] + f;
    double sn, cs;
    sincos(A.omega[b] * t, &sn, &cs);
    g += A.Xre[b] * cs + A.Xim[b] * sn;
  }
  A.gn[(long long)s * A.n_inst + i] = 2.0 * A.S * g;
}

int adjoint_step_launch(const AdjArgs& a, cudaStream_t st) {
  adjoint_step_kernel<<<a.n_tiles, 256, 0, st>>>(a);
  return (int)cudaGetLastError();
}

int probe_adjoint_launch(const ProbeAdjArgs& a, cudaStream_t st) {
  probe_adjoint_kernel<<<(a.n_inst + 127) / 128, 128, 0, st>>>(a);
  return (int)cudaGetLastError();
}

int loss_source_launch(const SourceAdjArgs& a, cudaStream_t st) {
  const int total = a.n_inst * a.steps;
  if (total == 0) return 0;
  loss_source_kernel<<<(total + 255) / 256, 256, 0, st>>>(a);
  return (int)cudaGetLastError();
}

}  // namespace gfdtd
