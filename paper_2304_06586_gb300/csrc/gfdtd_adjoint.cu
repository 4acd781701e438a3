// gfdtd_adjoint.cu -- reverse-time discrete adjoint of the batched step.
//
// For moving perturbation the step n maps (B^{n-1}, D^{n-1/2}) linearly to
// (B^n, D^{n+1/2}) (Sec. 4 with Table 1; the source adds a constant):
//   E'_k = se_k D_k - cb Bsum_k,   B'_j = a B_j + c B_up(j) + E'_j - E'_{j+1},
//   H'_j = sm_j B'_j - cb (D_j + D_{j+1}),   D'_k = a D_k + c D_up(k) + H'_{k-1} - H'_k,
// with E' = S E*, H' = S H*.  The reverse sweep applies the transpose, gathered
// per cell, to the adjoint fields (lB', lD') of (B^n, D^{n+1/2}):
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
#include <climits>

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

// Number of profile positions b in [0, np) with zq[b] <= xi, i.e. at or left
// of the node whose moving coordinate is xi = k 2^32 - off (binary search;
// cells beyond the first or last position take two loads).
__device__ __forceinline__ int positions_at_or_left(const long long* __restrict__ zq, int np, long long xi) {
  if (np == 0 || __ldg(zq) > xi) return 0;
  if (__ldg(zq + np - 1) <= xi) return np;
  int lo = 1, hi = np - 1;                    // zq[0] <= xi < zq[np - 1]
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (__ldg(zq + mid) <= xi) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// A non-negative 64-bit integer as FP32 from its two 32-bit halves (two 32-bit
// conversions and one FMA instead of a 64-bit conversion).
__device__ __forceinline__ float i64_to_f32(long long x) {
  return fmaf((float)(int)(x >> 32), 4294967296.0f, (float)(unsigned)x);
}

// ------------------------------------------------ time-blocked reverse steps
//
// adjoint_block_kernel transposes up to kAdjBlockSteps consecutive steps per
// launch (n = n_hi, n_hi - 1, ...).  A warp holds the adjoint fields of a
// window of 32 x kAdjCells cells of one instance in registers (lane l: cells
// base + 8 l .. base + 8 l + 7) and applies the gathered transpose above one
// step at a time, trading the ends of each lane's run with its neighbours by
// shuffles; only the tile's output range is stored at the end, where the
// margins keep it exact (adj_margin, adj_width).  Cells outside [0, nz) stay
// zero, as the forward's ghosts are.  D^{n-1/2} of each step comes from the
// segment's recomputation.  The probe term of step n (F_n = D_p se_p / S at
// level n+1/2, with dL/dF_n from loss_source_kernel) enters lD' of every
// window that holds the probe node, before the step, and its permittivity
// term once, from the tile whose output range holds the node.
// The permittivity gradient of the output cells adds up per lane over runs of
// one profile value, then per warp in shared memory over the values the
// window can meet in the launch, and reaches the FP64 gradient with one
// atomic per value and tile; a window that stays before the first profile
// position or after the last one over the whole launch has a single value,
// summed in registers.

constexpr int kAdjKeysW = 192;     // profile values a warp collects in shared memory

struct GradRun {
  int key;
  float acc;
};

// Hands a lane's run to the warp's accumulators (values kb .. kb + kAdjKeysW - 1)
// or, outside them, to the FP64 gradient.
__device__ __forceinline__ void grad_flush(GradRun& r, float* sacc, int kb, double* grad) {
  if (r.key >= 0 && r.acc != 0.0f) {
    const int slot = r.key - kb;
    if (slot >= 0 && slot < kAdjKeysW) atomicAdd(sacc + slot, r.acc);
    else atomicAdd(grad + r.key, (double)r.acc);
  }
  r.acc = 0.0f;
}
__device__ __forceinline__ void grad_add(GradRun& r, int key, float v, float* sacc, int kb, double* grad) {
  if (key != r.key) {
    grad_flush(r, sacc, kb, grad);
    r.key = key;
  }
  r.acc += v;
}

static_assert(kAdjBlockSteps <= 8, "cp_async_wait_upto covers up to 8 groups");

// The state of one tile of the time-blocked transpose between its setup and its store.
struct AdjTile {
  float LB[kAdjCells], LD[kAdjCells];   // lambda B, lambda D of the lane's cells
  int base, k0, x0, out_hi, nz;
  int kb, li, liH, ku;                  // gradient key base; position counts; single key (-1: none)
  float seu;                            // the single value's S/eps (ku >= 0)
  int kp, lp, cp;                       // probe node, its lane and cell (lp = -1: not in the window)
  bool probe_out;
  GradRun run;
  float gacc;                           // sum of lambdaE D over the output cells (ku >= 0)
};

// The reverse steps of one tile.  INSIDE: the window lies inside [0, nz), so no
// cell needs the zero of the domain's ghosts; UNI: one permittivity value over
// the window and the launch (key ku), whose gradient is -se^2 / S times the
// sum of lambdaE D over the output cells.
template <bool POS, bool INSIDE, bool UNI>
__device__ __forceinline__ void adjoint_steps(const AdjBlockArgs& A, const InstDev& I, int inst, AdjTile& T,
                                              float* sacc, float* sD, double* grad, int lane) {
  constexpr int C = kAdjCells;
  float (&LB)[C] = T.LB;
  float (&LD)[C] = T.LD;
  const int k0 = T.k0, nz = T.nz;
  const float a = I.a32, cc = I.c32, cb = I.cb32, S = (float)I.S, inv_S = (float)I.inv_S;
  const bool lin = (I.flags & F_LINEAR) != 0;
  const bool mu_const = (I.flags & F_MU_CONST) != 0;
  const long long dq = I.dq;
  const long long* __restrict__ zq = A.tb.zq + I.tab;
  const float2* __restrict__ tv = A.tb.tabE32 + I.tab;
  const int np = lin ? I.n : I.n - 1;
  // the lane's cells against the output range: all in, some in (a domain end), none
  const bool out_all = k0 >= T.x0 && k0 + C <= T.out_hi;
  const bool out_some = !out_all && k0 + C > T.x0 && k0 < T.out_hi;
  auto in = [&](int c) { return INSIDE || (unsigned)(k0 + c) < (unsigned)nz; };

  // D^{n-1/2} of every step of the launch (the forward's field after segment step m - 1),
  // copied asynchronously into this lane's part of the warp's buffer, one group per step
  float* myD = sD + lane * C;
  for (int s = 0; s < A.nsteps; ++s) {
    const float* src = A.dseg + (long long)(A.m_hi - 1 - s) * A.dseg_stride + I.off;
#pragma unroll
    for (int j = 0; j < C; j += 4) {
      const int kc = k0 + j;
      const bool ok = kc >= 0 && kc < I.nz_pad;
      cp_async16(myD + s * 32 * C + j, src + (ok ? kc : 0), ok);
    }
    cp_async_commit();
  }
  for (int s = 0; s < A.nsteps; ++s) {
    const int m = A.m_hi - s;                        // segment step transposed: n = n_seg + m
    const long long n = A.n_seg + m;
    float Dv[C];
    cp_async_wait_upto(A.nsteps - 1 - s);
#pragma unroll
    for (int j = 0; j < C; j += 4) {
      const float4 v = *reinterpret_cast<const float4*>(myD + s * 32 * C + j);
      Dv[j] = v.x;
      Dv[j + 1] = v.y;
      Dv[j + 2] = v.z;
      Dv[j + 3] = v.w;
    }

    // probe term of step n (level n+1/2) into lD'
    if (lane == T.lp) {
      const double g = A.gn[(long long)(m - 1) * A.n_inst + inst];
      if (g != 0.0) {
        const long long off = dq * (2 * n + 1);
        double se, y;
        node_coef<false, true>(I, A.tb, off, T.kp, se, y);
        const float add = (float)(g * se / I.S);
#pragma unroll
        for (int c = 0; c < C; ++c) LD[c] += (c == T.cp) ? add : 0.0f;
        if (T.probe_out) {
          // F = D / eps: dF/deps = -D / eps^2 = -D se^2 / S^2
          const double Dp = A.dseg[(long long)m * A.dseg_stride + I.off + T.kp];
          const double gE = g * (-Dp * se * se / (I.S * I.S));
          int i0, i1;
          double w0, w1;
          eps_weights(I, zq, ((long long)T.kp << 32) - off, i0, w0, i1, w1);
          atomicAdd(grad + i0, gE * w0);
          if (lin) atomicAdd(grad + i1, gE * w1);
        }
      }
    }

    // lH_j = lD'_{j+1} - lD'_j and lBt_j = lB'_j + sm_j lH_j
    const float dn1 = __shfl_down_sync(FULL, LD[0], 1);
    float lH[C], Tt[C];
    {
      float smv[C];
      if (mu_const) {
#pragma unroll
        for (int c = 0; c < C; ++c) smv[c] = I.sm32;
      } else {
        float tmp[C];
        lane_coefs<C, false, false, float>(I, A.tb, dq * (2 * n) - HALF_CELL, k0, T.liH, smv, tmp);
      }
#pragma unroll
      for (int c = 0; c < C; ++c) {
        lH[c] = in(c) ? (c + 1 < C ? LD[c + 1] : dn1) - LD[c] : 0.0f;
        Tt[c] = in(c) ? LB[c] + smv[c] * lH[c] : 0.0f;
      }
    }
    // lE_k = lBt_k - lBt_{k-1}
    const float tl1 = __shfl_up_sync(FULL, Tt[C - 1], 1);
    float lE[C];
#pragma unroll
    for (int c = 0; c < C; ++c) lE[c] = in(c) ? Tt[c] - (c > 0 ? Tt[c - 1] : tl1) : 0.0f;
    const float hl1 = __shfl_up_sync(FULL, lH[C - 1], 1);
    const float dl1 = __shfl_up_sync(FULL, LD[C - 1], 1);
    const float tn1 = __shfl_down_sync(FULL, Tt[0], 1);
    const float en1 = __shfl_down_sync(FULL, lE[0], 1);
    const float en2 = __shfl_down_sync(FULL, lE[1], 1);
    const float el1 = __shfl_up_sync(FULL, lE[C - 1], 1);

    // the permittivity at level n-1/2 of each cell, with the profile values it weighs
    const long long xi0 = ((long long)k0 << 32) - dq * (2 * n - 1);
    if (!UNI) {
      while (T.li < np && __ldg(zq + T.li) <= xi0) ++T.li;
      while (T.li > 0 && __ldg(zq + T.li - 1) > xi0) --T.li;
    }
    int idx = T.li;
    float nD[C], nB[C];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      float se, w1 = 0.0f;
      int key0 = T.ku, key1 = T.ku;
      if (UNI) {
        se = T.seu;
      } else {
        const long long xi = xi0 + ((long long)c << 32);
        while (idx < np && __ldg(zq + idx) <= xi) ++idx;
        if (lin) {
          float e;
          if (idx <= 0) {
            e = __ldg(tv).x;
            key0 = key1 = 0;
          } else if (idx >= np) {
            e = __ldg(tv + np - 1).x;
            key0 = key1 = np - 1;
          } else {
            const long long z0 = __ldg(zq + idx - 1), z1 = __ldg(zq + idx);
            w1 = quick_div(i64_to_f32(xi - z0), i64_to_f32(z1 - z0));
            const float e0 = __ldg(tv + idx - 1).x, e1 = __ldg(tv + idx).x;
            e = e0 + w1 * (e1 - e0);
            key0 = idx - 1;
            key1 = idx;
          }
          se = quick_div(S, e);
        } else {
          se = __ldg(tv + idx).x;
          key0 = key1 = idx;
        }
      }
      // lD_k = a lD'_k + c lD'_dn(k) - cb (lH_k + lH_{k-1}) + se_k lE_k
      const float ldn = POS ? (c + 1 < C ? LD[c + 1] : dn1) : (c > 0 ? LD[c - 1] : dl1);
      const float hm1 = c > 0 ? lH[c - 1] : hl1;
      nD[c] = in(c) ? a * LD[c] + cc * ldn - cb * (lH[c] + hm1) + se * lE[c] : 0.0f;
      // lB_j = a lBt_j + c lBt_dn(j) - cb (lE_{j+1} + lE_{j+2})  (v >= 0)
      //                                 - cb (lE_j + lE_{j-1})      (v < 0)
      if (POS) {
        const float tdn = c + 1 < C ? Tt[c + 1] : tn1;
        const float e1 = c + 1 < C ? lE[c + 1] : en1;
        const float e2 = c + 2 < C ? lE[c + 2] : (c + 2 == C ? en1 : en2);
        nB[c] = in(c) ? a * Tt[c] + cc * tdn - cb * (e1 + e2) : 0.0f;
      } else {
        const float tdn = c > 0 ? Tt[c - 1] : tl1;
        const float em1 = c > 0 ? lE[c - 1] : el1;
        nB[c] = in(c) ? a * Tt[c] + cc * tdn - cb * (lE[c] + em1) : 0.0f;
      }
      // dL/deps_k = lE_k (-S D_k / eps_k^2) = lE_k (-se^2 D_k / S), output cells only
      const bool out = out_all || (out_some && k0 + c >= T.x0 && k0 + c < T.out_hi);
      if (UNI) {
        if (out) T.gacc += lE[c] * Dv[c];
      } else if (out) {
        const float gE = lE[c] * (-se * se * Dv[c] * inv_S);
        grad_add(T.run, key0, gE * (1.0f - w1), sacc, T.kb, grad);
        grad_add(T.run, key1, gE * w1, sacc, T.kb, grad);
      }
    }
#pragma unroll
    for (int c = 0; c < C; ++c) {
      LB[c] = nB[c];
      LD[c] = nD[c];
    }
  }
}

template <bool POS>
__device__ __forceinline__ void adjoint_tile(const AdjBlockArgs& A, const InstDev& I, int inst, int x0,
                                             float* sacc, float* sD, double* grad, int lane) {
  constexpr int C = kAdjCells;
  AdjTile T;
  T.base = x0 - adj_margin(POS);
  T.k0 = T.base + C * lane;
  T.x0 = x0;
  T.nz = I.nz;
  T.out_hi = min(x0 + adj_width(POS), I.nz);          // output cells [x0, out_hi)
  const int base = T.base, k0 = T.k0, nz = T.nz;
  load_cells<float, float, C>(A.lBn + I.off, k0, I.nz_pad, T.LB);
  load_cells<float, float, C>(A.lDn + I.off, k0, I.nz_pad, T.LD);
#pragma unroll
  for (int c = 0; c < C; ++c) {   // (padding cells past nz are not necessarily written)
    const bool in = (unsigned)(k0 + c) < (unsigned)nz;
    T.LB[c] = in ? T.LB[c] : 0.0f;
    T.LD[c] = in ? T.LD[c] : 0.0f;
  }
  const bool lin = (I.flags & F_LINEAR) != 0;
  const long long dq = I.dq;
  const long long* __restrict__ zq = A.tb.zq + I.tab;
  const float2* __restrict__ tv = A.tb.tabE32 + I.tab;
  const int np = lin ? I.n : I.n - 1;                  // profile positions
  const long long n_hi = A.n_seg + A.m_hi, n_lo = n_hi - A.nsteps + 1;

  // a single permittivity value over the window and the launch (key ku), else ku = -1
  T.ku = -1;
  T.seu = 0.0f;
  {
    const int last = base + 32 * C - 1;
    const long long oa = dq * (2 * n_lo - 1), ob = dq * (2 * n_hi - 1);
    if (np == 0) {
      T.ku = 0;
    } else {
      const long long zf = __ldg(zq), zl = __ldg(zq + np - 1);
      if (last < node_of(zf, oa) && last < node_of(zf, ob)) T.ku = 0;
      else if (base >= node_of(zl, oa) && base >= node_of(zl, ob)) T.ku = lin ? np - 1 : np;
    }
    if (T.ku >= 0) {
      const float2 v = __ldg(tv + T.ku);
      T.seu = lin ? (float)I.S / v.x : v.x;
    }
  }
  T.kb = 0;
  T.li = 0;
  T.liH = 0;
  if (T.ku < 0) {
    // the smallest value the window meets in the launch: one below the count at its first cell
    const long long xa = ((long long)base << 32) - dq * (2 * n_lo - 1);
    const long long xb = ((long long)base << 32) - dq * (2 * n_hi - 1);
    T.kb = max(0, positions_at_or_left(zq, np, min(xa, xb)) - 1);
    for (int i = lane; i < kAdjKeysW; i += 32) sacc[i] = 0.0f;
    __syncwarp();
    T.li = positions_at_or_left(zq, np, ((long long)k0 << 32) - dq * (2 * n_hi - 1));
  }
  if (!(I.flags & F_MU_CONST)) T.liH = count_at_or_left(zq, np, dq * (2 * n_hi) - HALF_CELL, k0);
  // the probe
  T.kp = A.probe_node[inst];
  const bool probe_in = T.kp >= 0 && T.kp < nz && T.kp >= base && T.kp < base + 32 * C;
  T.probe_out = probe_in && T.kp >= x0 && T.kp < T.out_hi;
  T.lp = probe_in ? (T.kp - base) / C : -1;
  T.cp = probe_in ? (T.kp - base) % C : 0;
  T.run = GradRun{-1, 0.0f};
  T.gacc = 0.0f;

  const bool inside = base >= 0 && base + 32 * C <= nz;
  if (T.ku >= 0) {
    if (inside) adjoint_steps<POS, true, true>(A, I, inst, T, sacc, sD, grad, lane);
    else adjoint_steps<POS, false, true>(A, I, inst, T, sacc, sD, grad, lane);
  } else {
    if (inside) adjoint_steps<POS, true, false>(A, I, inst, T, sacc, sD, grad, lane);
    else adjoint_steps<POS, false, false>(A, I, inst, T, sacc, sD, grad, lane);
  }

  const int hi = min(x0 + adj_width(POS), I.nz_pad);
  store_cells<float, float, C>(A.lB + I.off, k0, x0, hi, T.LB);
  store_cells<float, float, C>(A.lD + I.off, k0, x0, hi, T.LD);
  if (T.ku >= 0) {
    // dL/deps = -se^2 / S times the sum of lambdaE D over the output cells and steps
    float g = T.gacc;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) g += __shfl_xor_sync(FULL, g, o);
    if (lane == 0 && g != 0.0f) atomicAdd(grad + T.ku, (double)g * (-(double)T.seu * T.seu / I.S));
  } else {
    grad_flush(T.run, sacc, T.kb, grad);
    __syncwarp();
    for (int i = lane; i < kAdjKeysW; i += 32)
      if (sacc[i] != 0.0f) atomicAdd(grad + T.kb + i, (double)sacc[i]);
    __syncwarp();
  }
}

__global__ void __launch_bounds__(128, 5) adjoint_block_kernel(const AdjBlockArgs A) {
  constexpr int WPB = 4;
  __shared__ float s_acc[WPB][kAdjKeysW];
  __shared__ __align__(16) float s_D[WPB][kAdjBlockSteps * 32 * kAdjCells];   // D rows of the warp's tile
  const int wib = __shfl_sync(FULL, (int)(threadIdx.x >> 5), 0), lane = threadIdx.x & 31;
  const int gw = blockIdx.x * WPB + wib, nw = gridDim.x * WPB;
  // (blocks add into different copies of the gradient, so that the many warps of one
  // uniform region do not all queue on the same profile value's atomics)
  double* gcopy = A.grad + (size_t)(blockIdx.x % A.grad_copies) * A.grad_stride;
  for (int t = gw; t < A.n_tiles; t += nw) {
    const int2 tl = A.tiles[t];
    const InstDev I = A.inst[tl.x];
    if (I.flags & F_POS) adjoint_tile<true>(A, I, tl.x, tl.y, s_acc[wib], s_D[wib], gcopy + I.tab, lane);
    else adjoint_tile<false>(A, I, tl.x, tl.y, s_acc[wib], s_D[wib], gcopy + I.tab, lane);
  }
}

int adjoint_block_launch(const AdjBlockArgs& a, int grid, cudaStream_t st) {
  adjoint_block_kernel<<<grid, 128, 0, st>>>(a);
  return (int)cudaGetLastError();
}

int adjoint_block_occupancy(int* blocks_per_sm) {
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(blocks_per_sm, adjoint_block_kernel, 128, 0);
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

__global__ void sum_copies_kernel(const double* __restrict__ copies, long long n_copies, long long stride,
                                  long long n, double* __restrict__ out) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double t = 0.0;
  for (long long c = 0; c < n_copies; ++c) t += copies[c * stride + i];
  out[i] = t;
}

int sum_copies_launch(const double* copies, long long n_copies, long long stride, long long n, double* out,
                      cudaStream_t st) {
  if (n == 0) return 0;
  sum_copies_kernel<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(copies, n_copies, stride, n, out);
  return (int)cudaGetLastError();
}

int loss_source_launch(const SourceAdjArgs& a, cudaStream_t st) {
  const int total = a.n_inst * a.steps;
  if (total == 0) return 0;
  loss_source_kernel<<<(total + 255) / 256, 256, 0, st>>>(a);
  return (int)cudaGetLastError();
}

}  // namespace gfdtd
