// gfdtd_block.cuh -- the batched time-block kernel of the generalized-FDTD
// engine and the device helpers it shares with the other kernels.
//
// The scheme (Sec. 4 of Deck-Leger et al., arXiv 2304.06586) advances, per
// step n and per cell, with E' = S E* and H' = S H*:
//
//   E'_k   = se_k D_k - cb_k Bsum_k                     Eq. Dconst_discr, Table 1 Ba/Bb
//            Bsum_k = B_{k-1} + B_{k-2} (v >= 0) or B_k + B_{k+1} (v < 0)
//   B_j   <- a B_j + c B_{j-1 | j+1} + E'_j - E'_{j+1}  Eq. Farad_discr, Table 1 dBa/dBb
//   H'_j   = sm_j B_j - cb_j (D_j + D_{j+1})            Eq. Bconst_discr, Table 1 Da/Db
//   D_k   <- a D_k + c D_{k-1 | k+1} + H'_{k-1} - H'_k  Eq. Ampere_discr, Table 1 dDa/dDb
//
// with a = 1 - |v| S, c = |v| S, se = S/eps (level n-1/2), sm = S/mu (level n)
// and cb = S v / 2 (moving matter: the per-node coefficients of the solved
// star relations).  Array index j of B is the half node j + 1/2.
//
// Every warp owns a tile of 32 x C consecutive cells of one instance held in
// registers (C per lane) and advances it TB steps before writing back,
// exchanging neighbour values with warp shuffles.  One step reaches 3 cells
// upwind and 1 downwind for v >= 0 (1 and 2 for v < 0), so a tile that loads
// its output range widened by that cone times TB needs no synchronisation
// with other tiles: the cone margins are recomputed by both neighbours.
// Tiles of all instances are spread over a persistent grid, one launch per
// time block, and the state ping-pongs between two buffers.
#pragma once

#include "gfdtd_internal.cuh"

#include <climits>

namespace gfdtd {

constexpr unsigned FULL = 0xffffffffu;
constexpr long long HALF_CELL = 2147483648LL;   // 2^31: half a cell in 32.32 fixed point

// ------------------------------------------------------------------ storage

template <typename T> struct Real { using type = float; };
template <> struct Real<double> { using type = double; };

__device__ __forceinline__ void unpack(uint4 u, float* x, float) {
  x[0] = __uint_as_float(u.x); x[1] = __uint_as_float(u.y);
  x[2] = __uint_as_float(u.z); x[3] = __uint_as_float(u.w);
}
__device__ __forceinline__ void unpack(uint4 u, float* x, __nv_bfloat16) {
  const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat162 h;
    *reinterpret_cast<unsigned*>(&h) = w[i];
    const float2 f = __bfloat1622float2(h);
    x[2 * i] = f.x; x[2 * i + 1] = f.y;
  }
}
__device__ __forceinline__ void unpack(uint4 u, float* x, __half) {
  const unsigned w[4] = {u.x, u.y, u.z, u.w};
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __half2 h;
    *reinterpret_cast<unsigned*>(&h) = w[i];
    const float2 f = __half22float2(h);
    x[2 * i] = f.x; x[2 * i + 1] = f.y;
  }
}
__device__ __forceinline__ void unpack(uint4 u, double* x, double) {
  x[0] = __hiloint2double((int)u.y, (int)u.x);
  x[1] = __hiloint2double((int)u.w, (int)u.z);
}

__device__ __forceinline__ uint4 pack(const float* x, float) {
  return make_uint4(__float_as_uint(x[0]), __float_as_uint(x[1]), __float_as_uint(x[2]),
                    __float_as_uint(x[3]));
}
__device__ __forceinline__ uint4 pack(const float* x, __nv_bfloat16) {
  unsigned w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __nv_bfloat162 h = __floats2bfloat162_rn(x[2 * i], x[2 * i + 1]);
    w[i] = *reinterpret_cast<const unsigned*>(&h);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ uint4 pack(const float* x, __half) {
  unsigned w[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const __half2 h = __floats2half2_rn(x[2 * i], x[2 * i + 1]);
    w[i] = *reinterpret_cast<const unsigned*>(&h);
  }
  return make_uint4(w[0], w[1], w[2], w[3]);
}
__device__ __forceinline__ uint4 pack(const double* x, double) {
  return make_uint4((unsigned)__double2loint(x[0]), (unsigned)__double2hiint(x[0]),
                    (unsigned)__double2loint(x[1]), (unsigned)__double2hiint(x[1]));
}

// Load cells [k0, k0 + C) of one instance; 16-byte chunks outside [0, nz_pad) read as zero.
template <typename T, typename R, int C>
__device__ __forceinline__ void load_cells(const T* __restrict__ p, int k0, int nz_pad, R (&x)[C]) {
  constexpr int V = 16 / sizeof(T);
  static_assert(C % V == 0, "a lane must hold whole 16-byte chunks");
#pragma unroll
  for (int j = 0; j < C / V; ++j) {
    const int kc = k0 + j * V;
    uint4 u = make_uint4(0u, 0u, 0u, 0u);
    if (kc >= 0 && kc < nz_pad) u = __ldg(reinterpret_cast<const uint4*>(p + kc));
    unpack(u, &x[j * V], T());
  }
}

// Store the chunks of cells [k0, k0 + C) that lie in [lo, hi).
template <typename T, typename R, int C>
__device__ __forceinline__ void store_cells(T* __restrict__ p, int k0, int lo, int hi,
                                            const R (&x)[C]) {
  constexpr int V = 16 / sizeof(T);
#pragma unroll
  for (int j = 0; j < C / V; ++j) {
    const int kc = k0 + j * V;
    if (kc >= lo && kc < hi) *reinterpret_cast<uint4*>(p + kc) = pack(&x[j * V], T());
  }
}

// ------------------------------------------------------------ material

// First node at or beyond a profile position zq when the frame has moved by
// `off` (units of 2^-32 cell): ceil((zq + off) / 2^32).  For integer nodes at
// half level h, off = dq h; for half nodes, off = dq h - 2^31.
__device__ __forceinline__ int node_of(long long zq, long long off) {
  return (int)((zq + off + 0xFFFFFFFFLL) >> 32);
}

// Number of profile positions b in [0, nb) with node_of(zq[b]) <= k (binary search).
__device__ __forceinline__ int count_at_or_left(const long long* __restrict__ zq, int nb,
                                                long long off, int k) {
  int lo = 0, hi = nb;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (node_of(__ldg(zq + mid), off) <= k) lo = mid + 1; else hi = mid;
  }
  return lo;
}

// Coefficients (x: S/eps or S/mu, y: coupling) of a LINEAR profile at node k,
// `idx` = number of knots at or left of k; evaluated in the arithmetic type R.
template <bool MATTER, bool ESIDE, typename R>
__device__ __forceinline__ void linear_coef(const InstDev& I, const long long* __restrict__ zq,
                                            const double2* __restrict__ raw, int idx, int k,
                                            long long off, R& cx, R& cy) {
  const int n = I.n;
  R e, m;
  if (idx <= 0) {
    const double2 v = __ldg(raw); e = (R)v.x; m = (R)v.y;
  } else if (idx >= n) {
    const double2 v = __ldg(raw + n - 1); e = (R)v.x; m = (R)v.y;
  } else {
    const long long z0 = __ldg(zq + idx - 1), z1 = __ldg(zq + idx);
    const long long xi = ((long long)k << 32) - off;
    const R wgt = (R)(xi - z0) / (R)(z1 - z0);
    const double2 v0 = __ldg(raw + idx - 1), v1 = __ldg(raw + idx);
    e = (R)v0.x + wgt * ((R)v1.x - (R)v0.x);
    m = (R)v0.y + wgt * ((R)v1.y - (R)v0.y);
  }
  const R S = (R)I.S;
  if (!MATTER) {
    cx = S / (ESIDE ? e : m);
    cy = (R)I.cb;
  } else {
    const R b = (R)I.beta, g = (R)1 - b * b;
    const R den = e * m - b * b;
    cx = S * g * (ESIDE ? m : e) / den;
    cy = (R)0.5 * S * b * g / den;
  }
}

// Coefficients at a single node (binary search): used by probes and the plain kernel.
template <bool MATTER, bool ESIDE, typename R>
__device__ __forceinline__ void node_coef(const InstDev& I, const Tables& tb, long long off, int k,
                                          R& cx, R& cy) {
  const long long* zq = tb.zq + I.tab;
  const double2* tv = (ESIDE ? tb.tabE : tb.tabH) + I.tab;
  if (I.flags & F_LINEAR) {
    const int idx = count_at_or_left(zq, I.n, off, k);
    linear_coef<MATTER, ESIDE>(I, zq, tv, idx, k, off, cx, cy);
    return;
  }
  const double2 v = __ldg(tv + count_at_or_left(zq, I.n - 1, off, k));
  cx = (R)v.x;
  cy = MATTER ? (R)v.y : (R)I.cb;
}

// Per-lane material of the run of C cells starting at k0 at one half level.
// `li` carries, between steps, the number of profile positions at or left of k0.
template <int C, bool MATTER, bool ESIDE, typename R>
__device__ __forceinline__ void lane_coefs(const InstDev& I, const Tables& tb, long long off,
                                           int k0, int& li, R (&cx)[C], R (&cy)[C]) {
  const long long* __restrict__ zq = tb.zq + I.tab;
  const double2* __restrict__ tv = (ESIDE ? tb.tabE : tb.tabH) + I.tab;
  if (I.flags & F_LINEAR) {
    const int nk = I.n;
    while (li < nk && node_of(__ldg(zq + li), off) <= k0) ++li;
    while (li > 0 && node_of(__ldg(zq + li - 1), off) > k0) --li;
    int idx = li;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int k = k0 + c;
      while (idx < nk && node_of(__ldg(zq + idx), off) <= k) ++idx;
      linear_coef<MATTER, ESIDE>(I, zq, tv, idx, k, off, cx[c], cy[c]);
    }
    return;
  }
  const int nl = I.n, nb = nl - 1;
  while (li < nb && node_of(__ldg(zq + li), off) <= k0) ++li;
  while (li > 0 && node_of(__ldg(zq + li - 1), off) > k0) --li;
  const int K1 = li < nb ? node_of(__ldg(zq + li), off) : INT_MAX;
  const int K2 = li + 1 < nb ? node_of(__ldg(zq + li + 1), off) : INT_MAX;
  const bool many = li + 2 < nb && node_of(__ldg(zq + li + 2), off) < k0 + C;
  if (!many) {
    // at most two layer boundaries inside this lane's cells
    const double2 w0 = __ldg(tv + li);
    const double2 w1 = __ldg(tv + min(li + 1, nl - 1));
    const double2 w2 = __ldg(tv + min(li + 2, nl - 1));
    const R v0x = (R)w0.x, v1x = (R)w1.x, v2x = (R)w2.x;
    const R v0y = (R)w0.y, v1y = (R)w1.y, v2y = (R)w2.y;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int k = k0 + c;
      cx[c] = k >= K2 ? v2x : (k >= K1 ? v1x : v0x);
      if (MATTER) cy[c] = k >= K2 ? v2y : (k >= K1 ? v1y : v0y);
    }
  } else {
    int idx = li;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int k = k0 + c;
      while (idx < nb && node_of(__ldg(zq + idx), off) <= k) ++idx;
      const double2 v = __ldg(tv + idx);
      cx[c] = (R)v.x;
      if (MATTER) cy[c] = (R)v.y;
    }
  }
}

template <int C, typename R>
__device__ __forceinline__ R pick(const R (&x)[C], int c) {
  R v = x[0];
#pragma unroll
  for (int j = 1; j < C; ++j) v = (c == j) ? x[j] : v;
  return v;
}

// ------------------------------------------------------------- one tile

template <int C, int TB, bool POS, bool MATTER, bool EDGE, typename T>
__device__ __forceinline__ void run_tile(const BlockArgs<T>& A, const InstDev& I, int x0, int W,
                                         long long n0) {
  using R = typename Real<T>::type;
  const int lane = threadIdx.x & 31;
  constexpr int L = POS ? 3 * TB : TB;   // upwind margin of the dependency cone
  const int base = x0 - L;
  const int k0 = base + lane * C;
  const int nz = I.nz;

  R B[C], D[C], X[C];
  load_cells<T, R, C>(A.Bin + I.off, k0, I.nz_pad, B);
  load_cells<T, R, C>(A.Din + I.off, k0, I.nz_pad, D);

  const R a = (R)I.a, cc = (R)I.c;
  const bool eps_const = (I.flags & F_EPS_CONST) != 0;
  const bool mu_const = (I.flags & F_MU_CONST) != 0;
  const long long dq = I.dq;
  const double2 e0 = __ldg(A.tb.tabE + I.tab), h0 = __ldg(A.tb.tabH + I.tab);
  const R se0 = (R)e0.x, sm0 = (R)h0.x;
  const R cbe0 = MATTER ? (R)e0.y : (R)I.cb, cbh0 = MATTER ? (R)h0.y : (R)I.cb;
  int liE = 0, liH = 0;
  if (!eps_const || !mu_const) {
    const int nb = (I.flags & F_LINEAR) ? I.n : I.n - 1;
    liE = count_at_or_left(A.tb.zq + I.tab, nb, dq * (2 * n0 + 1), k0);
    liH = count_at_or_left(A.tb.zq + I.tab, nb, dq * (2 * n0 + 2) - HALF_CELL, k0);
  }

  // sources and probes that touch this tile (bit masks over the instance's lists)
  unsigned smask = 0, pmask = 0;
  if (A.src_amp) {
    for (int q = 0; q < I.nsrc && q < 32; ++q) {
      const int node = A.srcs[I.src0 + q].node;
      if (node >= base && node < base + 32 * C) smask |= 1u << q;
    }
  }
  if (A.record) {
    for (int q = 0; q < I.nprb && q < 32; ++q) {
      const int node = A.prbs[I.prb0 + q].node;
      if (node >= x0 && node < x0 + W && node < nz) pmask |= 1u << q;
    }
  }

  for (int s = 0; s < A.nsteps; ++s) {
    const long long n = n0 + s + 1;   // B^{n-1} -> B^n, D^{n-1/2} -> D^{n+1/2}

    // ---- E'^{n-1/2} = se D - cb Bsum  (B at level n-1, material at level n-1/2)
    R bl1, bl2, br1;
    if (POS) {
      bl1 = __shfl_up_sync(FULL, B[C - 1], 1);
      bl2 = __shfl_up_sync(FULL, B[C - 2], 1);
    } else {
      br1 = __shfl_down_sync(FULL, B[0], 1);
    }
    {
      R se[C], cbe[C];
      if (!eps_const) {
        lane_coefs<C, MATTER, true>(I, A.tb, dq * (2 * n - 1), k0, liE, se, cbe);
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) { se[c] = se0; cbe[c] = cbe0; }
      }
#pragma unroll
      for (int c = 0; c < C; ++c) {
        R bs;
        if (POS) {
          const R b1 = c >= 1 ? B[c - 1] : bl1;
          const R b2 = c >= 2 ? B[c - 2] : (c == 1 ? bl1 : bl2);
          bs = b1 + b2;
        } else {
          bs = B[c] + (c + 1 < C ? B[c + 1] : br1);
        }
        X[c] = se[c] * D[c] - (MATTER ? cbe[c] : cbe0) * bs;
        if (EDGE) X[c] = ((unsigned)(k0 + c) < (unsigned)nz) ? X[c] : (R)0;
      }
    }

    // ---- B^n (upwind difference at level n-1)
    {
      const R er = __shfl_down_sync(FULL, X[0], 1);
      if (POS) {
#pragma unroll
        for (int c = C - 1; c >= 0; --c) {
          const R bu = c >= 1 ? B[c - 1] : bl1;
          const R en = c + 1 < C ? X[c + 1] : er;
          B[c] = a * B[c] + (cc * bu + (X[c] - en));
          if (EDGE) B[c] = ((unsigned)(k0 + c) < (unsigned)nz) ? B[c] : (R)0;
        }
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const R bu = c + 1 < C ? B[c + 1] : br1;
          const R en = c + 1 < C ? X[c + 1] : er;
          B[c] = a * B[c] + (cc * bu + (X[c] - en));
          if (EDGE) B[c] = ((unsigned)(k0 + c) < (unsigned)nz) ? B[c] : (R)0;
        }
      }
    }

    // ---- H'^n = sm B - cb (D_j + D_{j+1})  (D at level n-1/2, material at level n)
    const R dr = __shfl_down_sync(FULL, D[0], 1);
    {
      R sm[C], cbh[C];
      if (!mu_const) {
        lane_coefs<C, MATTER, false>(I, A.tb, dq * (2 * n) - HALF_CELL, k0, liH, sm, cbh);
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) { sm[c] = sm0; cbh[c] = cbh0; }
      }
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const R d1 = c + 1 < C ? D[c + 1] : dr;
        X[c] = sm[c] * B[c] - (MATTER ? cbh[c] : cbh0) * (D[c] + d1);
        if (EDGE) X[c] = ((unsigned)(k0 + c) < (unsigned)nz) ? X[c] : (R)0;
      }
    }

    // ---- D^{n+1/2} (upwind difference at level n-1/2)
    {
      const R hl = __shfl_up_sync(FULL, X[C - 1], 1);
      if (POS) {
        const R dl = __shfl_up_sync(FULL, D[C - 1], 1);
#pragma unroll
        for (int c = C - 1; c >= 0; --c) {
          const R du = c >= 1 ? D[c - 1] : dl;
          const R hp = c >= 1 ? X[c - 1] : hl;
          D[c] = a * D[c] + (cc * du + (hp - X[c]));
          if (EDGE) D[c] = ((unsigned)(k0 + c) < (unsigned)nz) ? D[c] : (R)0;
        }
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const R du = c + 1 < C ? D[c + 1] : dr;
          const R hp = c >= 1 ? X[c - 1] : hl;
          D[c] = a * D[c] + (cc * du + (hp - X[c]));
          if (EDGE) D[c] = ((unsigned)(k0 + c) < (unsigned)nz) ? D[c] : (R)0;
        }
      }
    }

    // ---- soft sources at t_{n+1/2}
    for (unsigned m = smask; m; m &= m - 1) {
      const int q = __ffs(m) - 1;
      const int rel = A.srcs[I.src0 + q].node - base;
      const R amp = (R)A.src_amp[(long long)(I.src0 + q) * A.chunk_stride + A.s0 + s];
      if (lane == rel / C) {
        const int cs = rel % C;
#pragma unroll
        for (int c = 0; c < C; ++c) D[c] += (c == cs) ? amp : (R)0;
      }
    }

    // ---- probes: physical E at level n+1/2 (Eq. const_1d; matter: E = E* + v Bbar)
    for (unsigned m = pmask; m; m &= m - 1) {
      const int q = __ffs(m) - 1;
      const int node = A.prbs[I.prb0 + q].node;
      const int rel = node - base;
      const int lp = rel / C, cp = rel % C;
      R bbar = (R)0;
      if (MATTER) {
        if (POS) {
          const R b1l = __shfl_up_sync(FULL, B[C - 1], 1);
          const R b2l = __shfl_up_sync(FULL, B[C - 2], 1);
          const R b1 = cp >= 1 ? pick(B, cp - 1) : b1l;
          const R b2 = cp >= 2 ? pick(B, cp - 2) : (cp == 1 ? b1l : b2l);
          bbar = (R)0.5 * (b1 + b2);
        } else {
          const R b1r = __shfl_down_sync(FULL, B[0], 1);
          const R b1 = cp + 1 < C ? pick(B, cp + 1) : b1r;
          bbar = (R)0.5 * (pick(B, cp) + b1);
        }
      }
      if (lane == lp) {
        R sep, cbp;
        node_coef<MATTER, true>(I, A.tb, dq * (2 * n + 1), node, sep, cbp);
        R F = pick(D, cp) * sep;
        if (MATTER) F += ((R)I.beta * (R)I.S - (R)2 * cbp) * bbar;
        A.samples[(long long)(I.prb0 + q) * A.chunk_stride + A.s0 + s] = (double)(F * (R)I.inv_S);
      }
    }
  }

  const int hi = min(x0 + W, I.nz_pad);
  store_cells<T, R, C>(A.Bout + I.off, k0, x0, hi, B);
  store_cells<T, R, C>(A.Dout + I.off, k0, x0, hi, D);
}

// Tile width (output cells) of a tile shape for one sign of v.
__host__ __device__ constexpr int tile_width(int C, int TB, bool pos) {
  return 32 * C - (pos ? 4 * TB : 3 * TB);
}

template <int C, int TB, bool MATTER, typename T>
__global__ void __launch_bounds__(128) block_kernel(const BlockArgs<T> A) {
  const int warps_per_block = blockDim.x >> 5;
  const int gw = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const int nw = gridDim.x * warps_per_block;
  const long long n0 = *A.n_done + A.s0;
  for (int t = gw; t < A.n_tiles; t += nw) {
    const int2 tl = A.tiles[t];
    const InstDev I = A.inst[tl.x];
    const int x0 = tl.y;
    if (I.flags & F_POS) {
      constexpr int W = tile_width(C, TB, true);
      const int base = x0 - 3 * TB;
      if (base < 0 || base + 32 * C > I.nz) run_tile<C, TB, true, MATTER, true>(A, I, x0, W, n0);
      else run_tile<C, TB, true, MATTER, false>(A, I, x0, W, n0);
    } else {
      constexpr int W = tile_width(C, TB, false);
      const int base = x0 - TB;
      if (base < 0 || base + 32 * C > I.nz) run_tile<C, TB, false, MATTER, true>(A, I, x0, W, n0);
      else run_tile<C, TB, false, MATTER, false>(A, I, x0, W, n0);
    }
  }
}

template <int C, int TB, bool MATTER, typename T>
int launch_block_shape(const void* args, int grid, int block, cudaStream_t st) {
  block_kernel<C, TB, MATTER, T><<<grid, block, 0, st>>>(*static_cast<const BlockArgs<T>*>(args));
  return (int)cudaGetLastError();
}

template <int C, int TB, bool MATTER, typename T>
int occupancy_block_shape(int block, int* nb) {
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, block_kernel<C, TB, MATTER, T>,
                                                            block, 0);
}

}  // namespace gfdtd
