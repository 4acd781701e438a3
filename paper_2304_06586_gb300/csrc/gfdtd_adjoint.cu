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
template <typename W>
__device__ __forceinline__ void eps_weights(const InstDev& I, const long long* zq, long long xi,
                                            int& i0, W& w0, int& i1, W& w1) {
  if (!(I.flags & F_LINEAR)) {
    int lo = 0, hi = I.n - 1;                 // count of boundaries <= xi
    while (lo < hi) { const int mid = (lo + hi) >> 1; if (__ldg(zq + mid) <= xi) lo = mid + 1; else hi = mid; }
    i0 = lo; w0 = 1; i1 = lo; w1 = 0;
    return;
  }
  const int n = I.n;
  if (xi <= __ldg(zq)) { i0 = i1 = 0; w0 = 1; w1 = 0; return; }
  if (xi >= __ldg(zq + n - 1)) { i0 = i1 = n - 1; w0 = 1; w1 = 0; return; }
  int lo = 0, hi = n;                         // last knot <= xi
  while (hi - lo > 1) { const int mid = (lo + hi) >> 1; if (__ldg(zq + mid) <= xi) lo = mid; else hi = mid; }
  const W w = (W)(xi - __ldg(zq + lo)) / (W)(__ldg(zq + lo + 1) - __ldg(zq + lo));
  i0 = lo; w0 = (W)1 - w; i1 = lo + 1; w1 = w;
}

// Sum v over the lanes of the warp that share `key` (keys are non-decreasing
// across lanes); returns whether this lane is its segment's first, which then
// holds the sum.
__device__ __forceinline__ bool segment_sum(int& key, double& v, bool active) {
  const int lane = threadIdx.x & 31;
  if (!active) key = -1 - lane;               // inactive lanes form singleton segments
  for (int o = 1; o < 32; o <<= 1) {
    const double t = __shfl_down_sync(FULL, v, o);
    const int tk = __shfl_down_sync(FULL, key, o);
    if (lane + o < 32 && tk == key) v += t;
  }
  const int prev = __shfl_up_sync(FULL, key, 1);
  return active && (lane == 0 || prev != key) && v != 0.0;
}

constexpr int kAdjCells = 256;   // cells per block (one per thread)
constexpr int kAdjKeys = 512;    // profile values one block can reduce in shared memory

// One block transposes the step for 256 consecutive cells of one instance, in
// FP32 like the forward step; the permittivity gradient is summed per warp
// segment, then per block in shared memory, and added to the FP64 gradient
// with one atomic per profile value per block.
__global__ void __launch_bounds__(kAdjCells) adjoint_step_kernel(const AdjArgs A) {
  __shared__ float s_lb[kAdjCells + 8], s_ld[kAdjCells + 8];   // cells x0 - 2 .. x0 + 259
  __shared__ double s_g[kAdjKeys];
  __shared__ int s_key[2];
  const int2 tl = A.tiles[blockIdx.x];
  const InstDev I = A.inst[tl.x];
  const int x0 = tl.y, nz = I.nz, tid = threadIdx.x;
  const float* __restrict__ lBn = A.lBn + I.off;
  const float* __restrict__ lDn = A.lDn + I.off;
  for (int i = tid; i < kAdjCells + 6; i += kAdjCells) {
    const int j = x0 - 2 + i;
    const bool in = j >= 0 && j < nz;
    s_lb[i] = in ? lBn[j] : 0.0f;
    s_ld[i] = in ? lDn[j] : 0.0f;
  }
  for (int i = tid; i < kAdjKeys; i += kAdjCells) s_g[i] = 0.0;
  const int k = x0 + tid;
  const bool valid = k < nz;
  const bool pos = (I.flags & F_POS) != 0;
  const float a = I.a32, c = I.c32, cb = I.cb32;
  const long long n = A.n;
  const long long offH = I.dq * (2 * n) - HALF_CELL, offE = I.dq * (2 * n - 1);
  const bool mu_const = (I.flags & F_MU_CONST) != 0;
  auto in = [&](int j) { return j >= 0 && j < nz; };
  auto LB = [&](int j) -> float { return s_lb[j - x0 + 2]; };   // zero outside [0, nz)
  auto LD = [&](int j) -> float { return s_ld[j - x0 + 2]; };
  auto sm = [&](int j) -> float {
    if (mu_const) return I.sm32;
    float x, y;
    node_coef<false, false>(I, A.tb, offH, j, x, y);
    return x;
  };
  auto lH = [&](int j) -> float { return in(j) ? LD(j + 1) - LD(j) : 0.0f; };
  auto lBt = [&](int j) -> float { return in(j) ? LB(j) + sm(j) * lH(j) : 0.0f; };
  __syncthreads();

  int key0 = 0, key1 = 0;
  double g0 = 0.0, g1 = 0.0;
  if (valid) {
    float se, cbx;
    node_coef<false, true>(I, A.tb, offE, k, se, cbx);
    float lDk, lBk, lEk;
    if (pos) {
      const float tm1 = lBt(k - 1), t0 = lBt(k), t1 = lBt(k + 1), t2 = lBt(k + 2);
      lEk = t0 - tm1;
      const float lE1 = in(k + 1) ? t1 - t0 : 0.0f, lE2 = in(k + 2) ? t2 - t1 : 0.0f;
      lDk = a * LD(k) + c * LD(k + 1) - cb * (lH(k) + lH(k - 1)) + se * lEk;
      lBk = a * t0 + c * t1 - cb * (lE1 + lE2);
    } else {
      const float tm2 = lBt(k - 2), tm1 = lBt(k - 1), t0 = lBt(k);
      lEk = t0 - tm1;
      const float lEm1 = in(k - 1) ? tm1 - tm2 : 0.0f;
      lDk = a * LD(k) + c * LD(k - 1) - cb * (lH(k) + lH(k - 1)) + se * lEk;
      lBk = a * t0 + c * tm1 - cb * (lEk + lEm1);
    }
    A.lD[I.off + k] = lDk;
    A.lB[I.off + k] = lBk;
    // dL/deps_k = lE_k (-S D_k / eps_k^2) = lE_k (-se^2 D_k / S)
    const float gE = lEk * (-se * se * A.Dold[I.off + k] * (float)I.inv_S);
    float w0, w1;
    eps_weights(I, A.tb.zq + I.tab, ((long long)k << 32) - offE, key0, w0, key1, w1);
    g0 = (double)(gE * w0);
    g1 = (double)(gE * w1);
    if (tid == 0) s_key[0] = key0;
    if (tid == kAdjCells - 1 || k + 1 == nz) s_key[1] = key1;   // keys grow with k
  }
  __syncthreads();
  double* grad = A.grad + I.tab;
  const int kmin = s_key[0], span = s_key[1] - kmin + 1;
  const bool lin = (I.flags & F_LINEAR) != 0;
  const bool h0 = segment_sum(key0, g0, valid);
  const bool h1 = segment_sum(key1, g1, valid && lin);
  if (span <= kAdjKeys) {
    if (h0) atomicAdd(&s_g[key0 - kmin], g0);
    if (h1) atomicAdd(&s_g[key1 - kmin], g1);
    __syncthreads();
    for (int i = tid; i < span; i += kAdjCells)
      if (s_g[i] != 0.0) atomicAdd(grad + kmin + i, s_g[i]);
  } else {
    if (h0) atomicAdd(grad + key0, g0);
    if (h1) atomicAdd(grad + key1, g1);
  }
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
