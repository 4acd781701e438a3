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

// The FP64 or the FP32 copy of an instance coefficient, whichever R is (the FP32
// copies of a, c and cb are rounded so that a + c = 1 and c = 2 |cb| hold exactly).
template <typename R> __device__ __forceinline__ R coef(double d, float f);
template <> __device__ __forceinline__ float coef<float>(double, float f) { return f; }
template <> __device__ __forceinline__ double coef<double>(double d, float) { return d; }


// First node at or beyond a profile position zq when the frame has moved by
// `off` (units of 2^-32 cell): ceil((zq + off) / 2^32).  For integer nodes at
// half level h, off = dq h; for half nodes, off = dq h - 2^31.
__device__ __forceinline__ int node_of(long long zq, long long off) {
  return (int)((zq + off + 0xFFFFFFFFLL) >> 32);
}

// Graded absorbing layers of width W = I.abs_w at both domain ends (an option
// of this library; the paper is silent on the ends): a field sample at
// position x (D_k: x = k, B_k: x = k + 1/2) is multiplied right after its
// update by exp(-sigma d^2), d = (W - x) / W left of W, (x - (nz - 1 - W)) / W
// right of nz - 1 - W, else 0.
template <typename R>
__device__ __forceinline__ R absorb_factor(const InstDev& I, R x) {
  const R W = (R)I.abs_w, right = (R)(I.nz - 1) - W;
  R d = 0;
  if (x < W) d = (W - x) / W;
  else if (x > right) d = (x - right) / W;
  return exp(-(R)I.abs_sigma * d * d);
}
// Whether the window [base, base + span) reaches an absorbing layer.
__host__ __device__ inline bool window_absorbs(const InstDev& I, long long base, long long span) {
  return I.abs_w > 0 && (base < I.abs_w + 1 || base + span > I.nz - 2 - I.abs_w);
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
                                            const typename TabOf<R>::V* __restrict__ raw, int idx,
                                            int k, long long off, R& cx, R& cy) {
  const int n = I.n;
  R e, m;
  if (idx <= 0) {
    const auto v = __ldg(raw); e = v.x; m = v.y;
  } else if (idx >= n) {
    const auto v = __ldg(raw + n - 1); e = v.x; m = v.y;
  } else {
    const long long z0 = __ldg(zq + idx - 1), z1 = __ldg(zq + idx);
    const long long xi = ((long long)k << 32) - off;
    const R wgt = (R)(xi - z0) / (R)(z1 - z0);
    const auto v0 = __ldg(raw + idx - 1), v1 = __ldg(raw + idx);
    e = v0.x + wgt * (v1.x - v0.x);
    m = v0.y + wgt * (v1.y - v0.y);
  }
  const R S = (R)I.S;
  if (!MATTER) {
    cx = S / (ESIDE ? e : m);
    cy = coef<R>(I.cb, I.cb32);
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
  const auto* tv = TabOf<R>::get(tb, ESIDE) + I.tab;
  if (I.flags & F_LINEAR) {
    const int idx = count_at_or_left(zq, I.n, off, k);
    linear_coef<MATTER, ESIDE>(I, zq, tv, idx, k, off, cx, cy);
    return;
  }
  const auto v = __ldg(tv + count_at_or_left(zq, I.n - 1, off, k));
  cx = v.x;
  cy = MATTER ? v.y : coef<R>(I.cb, I.cb32);
}

// Per-lane material of the run of C cells starting at k0 at one half level.
// `li` carries, between steps, the number of profile positions at or left of k0.
// A 64-bit fixed-point difference in the arithmetic type: FP32 from the two
// 32-bit halves (two 32-bit conversions and an FMA; a 64-bit conversion is far
// slower), FP64 directly.
template <typename R> __device__ __forceinline__ R fixed_to_real(long long x);
template <> __device__ __forceinline__ float fixed_to_real<float>(long long x) {
  return fmaf((float)(int)(x >> 32), 4294967296.0f, (float)(unsigned)x);
}
template <> __device__ __forceinline__ double fixed_to_real<double>(long long x) { return (double)x; }

template <typename R> __device__ __forceinline__ R quick_div(R x, R y) { return x / y; }
template <> __device__ __forceinline__ float quick_div<float>(float x, float y) { return __fdividef(x, y); }

// The linear piece of a LINEAR profile between knots j-1 and j (j knots at or
// left; constant beyond the end knots) as (eps, mu) = alpha + beta t, with t in
// cells from the moving coordinate xi.
template <typename R, typename V>
__device__ __forceinline__ void lin_piece(const long long* __restrict__ zq, const V* __restrict__ raw, int nk,
                                          int j, long long xi, R& ae, R& be, R& am, R& bm) {
  if (j <= 0 || j >= nk) {
    const auto v = __ldg(raw + (j <= 0 ? 0 : nk - 1));
    ae = v.x; am = v.y; be = bm = (R)0;
    return;
  }
  const long long z0 = __ldg(zq + j - 1), z1 = __ldg(zq + j);
  const auto v0 = __ldg(raw + j - 1), v1 = __ldg(raw + j);
  const R inv = quick_div((R)1, fixed_to_real<R>(z1 - z0));
  const R w = fixed_to_real<R>(xi - z0) * inv, dw = (R)4294967296.0 * inv;
  const R de = (R)v1.x - (R)v0.x, dm = (R)v1.y - (R)v0.y;
  ae = (R)v0.x + w * de; be = dw * de;
  am = (R)v0.y + w * dm; bm = dw * dm;
}

// Coefficients (x: S/eps or S/mu, y: coupling) from the interpolated (eps, mu).
template <bool MATTER, bool ESIDE, typename R>
__device__ __forceinline__ void coef_of(R S, R beta, R cb, R e, R m, R& cx, R& cy) {
  if (!MATTER) {
    cx = quick_div(S, ESIDE ? e : m);
    cy = cb;
  } else {
    const R g = (R)1 - beta * beta;
    const R inv = quick_div((R)1, e * m - beta * beta);
    cx = S * g * (ESIDE ? m : e) * inv;
    cy = (R)0.5 * S * beta * g * inv;
  }
}

// The material coefficients (x: S/eps or S/mu, y: coupling; y is not formed for
// layers of a moving perturbation) of a lane's C cells k0 .. k0 + C - 1 at one
// level, handed to f(c, x, y) cell by cell as they are formed, so that the
// caller's update uses each at once and no per-cell array of them is kept.
template <int C, bool MATTER, bool ESIDE, typename R, typename F>
__device__ __forceinline__ void lane_apply(const InstDev& I, const Tables& tb, long long off,
                                           int k0, int& li, F&& f) {
  const long long* __restrict__ zq = tb.zq + I.tab;
  const auto* __restrict__ tv = TabOf<R>::get(tb, ESIDE) + I.tab;
  if (I.flags & F_LINEAR) {
    // eps and mu are linear between knots, so over a lane's cells they are a
    // few linear pieces in the cell index: each piece costs one evaluation per
    // lane, each cell an FMA and a division.
    const int nk = I.n;
    while (li < nk && node_of(__ldg(zq + li), off) <= k0) ++li;
    while (li > 0 && node_of(__ldg(zq + li - 1), off) > k0) --li;
    const R S = (R)I.S, beta = (R)I.beta, cb = coef<R>(I.cb, I.cb32);
    const long long xi0 = ((long long)k0 << 32) - off;
    const int K1 = li < nk ? node_of(__ldg(zq + li), off) : INT_MAX;
    const int K2 = li + 1 < nk ? node_of(__ldg(zq + li + 1), off) : INT_MAX;
    if (K2 >= k0 + C) {
      // at most one knot among the lane's cells: the piece left of it from
      // cell k0, the piece right of it from its first cell K1
      R aeL, beL, amL, bmL, aeR = 0, beR = 0, amR = 0, bmR = 0, mR = 0;
      lin_piece<R>(zq, tv, nk, li, xi0, aeL, beL, amL, bmL);
      if (K1 < k0 + C) {
        lin_piece<R>(zq, tv, nk, li + 1, xi0 + ((long long)(K1 - k0) << 32), aeR, beR, amR, bmR);
        mR = (R)(K1 - k0);
      }
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const bool r = k0 + c >= K1;
        const R t = (R)c - (r ? mR : (R)0);
        const R e = (r ? aeR : aeL) + (r ? beR : beL) * t;
        const R m = (r ? amR : amL) + (r ? bmR : bmL) * t;
        R x, y;
        coef_of<MATTER, ESIDE>(S, beta, cb, e, m, x, y);
        f(c, x, y);
      }
    } else {
      // several knots among the lane's cells: walk them cell by cell
      int idx = li;
      R ae, be, am, bm, t0 = 0;
      lin_piece<R>(zq, tv, nk, idx, xi0, ae, be, am, bm);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const long long xi = xi0 + ((long long)c << 32);
        if (idx < nk && __ldg(zq + idx) <= xi) {
          do ++idx; while (idx < nk && __ldg(zq + idx) <= xi);
          lin_piece<R>(zq, tv, nk, idx, xi, ae, be, am, bm);
          t0 = (R)c;
        }
        const R t = (R)c - t0;
        R x, y;
        coef_of<MATTER, ESIDE>(S, beta, cb, ae + be * t, am + bm * t, x, y);
        f(c, x, y);
      }
    }
    return;
  }
  const int nl = I.n, nb = nl - 1;
  while (li < nb && node_of(__ldg(zq + li), off) <= k0) ++li;
  while (li > 0 && node_of(__ldg(zq + li - 1), off) > k0) --li;
  const int K1 = li < nb ? node_of(__ldg(zq + li), off) : INT_MAX;
  const auto v0 = __ldg(tv + li);
  const auto v1 = __ldg(tv + min(li + 1, nl - 1));
  if (I.minw > C) {
    // layers wider than a lane's run: at most one boundary among its cells
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const bool past = k0 + c >= K1;
      f(c, (R)(past ? v1.x : v0.x), MATTER ? (R)(past ? v1.y : v0.y) : (R)0);
    }
    return;
  }
  const int K2 = li + 1 < nb ? node_of(__ldg(zq + li + 1), off) : INT_MAX;
  const bool many = li + 2 < nb && node_of(__ldg(zq + li + 2), off) < k0 + C;
  if (!many) {
    // at most two layer boundaries among this lane's cells
    const auto v2 = __ldg(tv + min(li + 2, nl - 1));
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int k = k0 + c;
      f(c, (R)(k >= K2 ? v2.x : (k >= K1 ? v1.x : v0.x)),
        MATTER ? (R)(k >= K2 ? v2.y : (k >= K1 ? v1.y : v0.y)) : (R)0);
    }
  } else {
    int idx = li;
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const int k = k0 + c;
      while (idx < nb && node_of(__ldg(zq + idx), off) <= k) ++idx;
      const auto v = __ldg(tv + idx);
      f(c, (R)v.x, MATTER ? (R)v.y : (R)0);
    }
  }
}

// The same coefficients stored per cell.
template <int C, bool MATTER, bool ESIDE, typename R>
__device__ __forceinline__ void lane_coefs(const InstDev& I, const Tables& tb, long long off,
                                           int k0, int& li, R (&cx)[C], R (&cy)[C]) {
  lane_apply<C, MATTER, ESIDE, R>(I, tb, off, k0, li, [&](int c, R x, R y) {
    cx[c] = x;
    cy[c] = y;
  });
}

template <int C, typename R>
__device__ __forceinline__ R pick(const R (&x)[C], int c) {
  R v = x[0];
#pragma unroll
  for (int j = 1; j < C; ++j) v = (c == j) ? x[j] : v;
  return v;
}

// ------------------------------------------------------------- one tile

// Kahan-compensated addition x += d with compensation cmp (F32_KAHAN tier).
template <typename R>
__device__ __forceinline__ void kahan_add(R& x, R& cmp, R d) {
  const R y = d - cmp;
  const R t = x + y;
  cmp = (t - x) - y;
  x = t;
}

// Which sides of a window [base, base + span) see a single material value over
// a launch of nsteps steps from n0 (E side: integer nodes at half levels
// 2n - 1; H side: half nodes at levels 2n): a uniform side of the instance, or
// a window that lies, over the whole launch, before the first profile position
// or after the last one (positions move monotonically, so the launch's first
// and last levels decide), with the table entry of that value in rE / rH.
// (Layers tables hold the coefficients themselves; a linear moving-matter
// profile would need them formed from (eps, mu), so it is never uniform here.)
__device__ __forceinline__ void uniform_sides(const InstDev& I, const Tables& tb, int base, int span, long long n0,
                                              int nsteps, bool& eps_const, bool& mu_const, int& rE, int& rH) {
  eps_const = (I.flags & F_EPS_CONST) != 0;
  mu_const = (I.flags & F_MU_CONST) != 0;
  rE = rH = 0;
  const bool lin = (I.flags & F_LINEAR) != 0;
  const int np = lin ? I.n : I.n - 1;                  // profile positions
  if ((!(I.flags & F_MATTER) || !lin) && np > 0 && (!eps_const || !mu_const)) {
    const long long* __restrict__ zq = tb.zq + I.tab;
    const long long zf = __ldg(zq), zl = __ldg(zq + np - 1);
    const int last = base + span - 1;
    const long long dq = I.dq;
    auto one_side = [&](long long off_a, long long off_b, int& r) {
      if (last < node_of(zf, off_a) && last < node_of(zf, off_b)) { r = 0; return true; }
      if (base >= node_of(zl, off_a) && base >= node_of(zl, off_b)) { r = lin ? np - 1 : np; return true; }
      return false;
    };
    const long long n1 = n0 + 1, n2 = n0 + nsteps;
    if (!eps_const && one_side(dq * (2 * n1 - 1), dq * (2 * n2 - 1), rE)) eps_const = true;
    if (!mu_const && one_side(dq * (2 * n1) - HALF_CELL, dq * (2 * n2) - HALF_CELL, rH)) mu_const = true;
  }
}

template <int C, int TB, bool POS, bool MATTER, bool EDGE, typename T, bool KAHAN = false>
__device__ __forceinline__ void run_tile(const BlockArgs<T>& A, const InstDev& I, int x0, int W,
                                         long long n0) {
  using R = typename Real<T>::type;
  const int lane = threadIdx.x & 31;
  constexpr int L = tile_margin(TB, POS, 16 / sizeof(T));   // x0 - base
  const int base = x0 - L;
  const int k0 = base + lane * C;
  const int nz = I.nz;

  R B[C], D[C], X[C];
  load_cells<T, R, C>(A.Bin + I.off, k0, I.nz_pad, B);
  load_cells<T, R, C>(A.Din + I.off, k0, I.nz_pad, D);
  R cBv[KAHAN ? C : 1], cDv[KAHAN ? C : 1];
  if constexpr (KAHAN) {
    load_cells<T, R, KAHAN ? C : 1>(A.cBin + I.off, k0, I.nz_pad, cBv);
    load_cells<T, R, KAHAN ? C : 1>(A.cDin + I.off, k0, I.nz_pad, cDv);
  }

  const R a = coef<R>(I.a, I.a32), cc = coef<R>(I.c, I.c32);
  const bool damp = window_absorbs(I, base, 32 * C);   // the tile reaches an absorbing layer
  bool eps_const, mu_const;
  int rE, rH;                                          // table entries of the uniform values
  uniform_sides(I, A.tb, base, 32 * C, n0, A.nsteps, eps_const, mu_const, rE, rH);
  const long long dq = I.dq;
  const bool lin = (I.flags & F_LINEAR) != 0;
  const auto e0 = __ldg(TabOf<R>::get(A.tb, true) + I.tab + rE);
  const auto h0 = __ldg(TabOf<R>::get(A.tb, false) + I.tab + rH);
  // (uniform values: LINEAR tables hold raw (eps, mu), LAYERS tables the coefficients)
  const R se0 = lin ? (R)I.S / e0.x : e0.x, sm0 = lin ? (R)I.S / h0.y : h0.x;
  const R cbe0 = MATTER ? e0.y : coef<R>(I.cb, I.cb32), cbh0 = MATTER ? h0.y : coef<R>(I.cb, I.cb32);
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
  // one-way sources whose correction cells (node - 2 .. node + 1) lie in this window
  unsigned tmask = 0;
  if (A.n_tfsf > 0) {
    for (int q = 0; q < I.ntf && q < 32; ++q) {
      const int node = A.tfsf[I.tf0 + q].node;
      if (node + 1 >= base && node - 2 < base + 32 * C) tmask |= 1u << q;
    }
  }
  // adds the one-way sources' corrections of this step to the cells first .. first + n - 1
  // (corrections j0 .. j0 + n - 1 of the step's record)
  auto tfsf_add = [&](R (&F)[C], int s, int first_off, int j0, int n) {
    for (unsigned m = tmask; m; m &= m - 1) {
      const int q = I.tf0 + __ffs(m) - 1;
      const int node = A.tfsf[q].node;
      const double* cr = A.tf_corr + ((long long)q * A.chunk_stride + A.s0 + s) * kTfsfCorr + j0;
      for (int j = 0; j < n; ++j) {
        const int k = node + first_off + j, rel = k - base;
        if (k >= 0 && k < nz && rel >= 0 && rel < 32 * C && lane == rel / C) {
          const R v = (R)cr[j];
          const int cs = rel % C;
#pragma unroll
          for (int c = 0; c < C; ++c) F[c] += (c == cs) ? v : (R)0;
        }
      }
    }
  };

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
      auto upd = [&](int c, R se, R cbe) {
        R bs;
        if (POS) {
          const R b1 = c >= 1 ? B[c - 1] : bl1;
          const R b2 = c >= 2 ? B[c - 2] : (c == 1 ? bl1 : bl2);
          bs = b1 + b2;
        } else {
          bs = B[c] + (c + 1 < C ? B[c + 1] : br1);
        }
        X[c] = se * D[c] - (MATTER ? cbe : cbe0) * bs;
        if (EDGE) X[c] = ((unsigned)(k0 + c) < (unsigned)nz) ? X[c] : (R)0;
      };
      if (!eps_const) {
        lane_apply<C, MATTER, true, R>(I, A.tb, dq * (2 * n - 1), k0, liE, upd);
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) upd(c, se0, cbe0);
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
          if (KAHAN) kahan_add(B[c], cBv[KAHAN ? c : 0], (X[c] - en) + cc * (bu - B[c]));
          else B[c] = a * B[c] + (cc * bu + (X[c] - en));
          if (EDGE) B[c] = ((unsigned)(k0 + c) < (unsigned)nz) ? B[c] : (R)0;
        }
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const R bu = c + 1 < C ? B[c + 1] : br1;
          const R en = c + 1 < C ? X[c + 1] : er;
          if (KAHAN) kahan_add(B[c], cBv[KAHAN ? c : 0], (X[c] - en) + cc * (bu - B[c]));
          else B[c] = a * B[c] + (cc * bu + (X[c] - en));
          if (EDGE) B[c] = ((unsigned)(k0 + c) < (unsigned)nz) ? B[c] : (R)0;
        }
      }
    }

    if (damp) {   // absorbing layers: B^n at x = k + 1/2
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const R g = absorb_factor<R>(I, (R)(k0 + c) + (R)0.5);
        B[c] *= g;
        if constexpr (KAHAN) cBv[c] *= g;
      }
    }
    if (tmask) tfsf_add(B, s, -2, 0, 4);   // one-way sources: B at node - 2 .. node + 1

    // ---- H'^n = sm B - cb (D_j + D_{j+1})  (D at level n-1/2, material at level n)
    const R dr = __shfl_down_sync(FULL, D[0], 1);
    {
      auto upd = [&](int c, R sm, R cbh) {
        const R d1 = c + 1 < C ? D[c + 1] : dr;
        X[c] = sm * B[c] - (MATTER ? cbh : cbh0) * (D[c] + d1);
        if (EDGE) X[c] = ((unsigned)(k0 + c) < (unsigned)nz) ? X[c] : (R)0;
      };
      if (!mu_const) {
        lane_apply<C, MATTER, false, R>(I, A.tb, dq * (2 * n) - HALF_CELL, k0, liH, upd);
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) upd(c, sm0, cbh0);
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
          if (KAHAN) kahan_add(D[c], cDv[KAHAN ? c : 0], (hp - X[c]) + cc * (du - D[c]));
          else D[c] = a * D[c] + (cc * du + (hp - X[c]));
          if (EDGE) D[c] = ((unsigned)(k0 + c) < (unsigned)nz) ? D[c] : (R)0;
        }
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const R du = c + 1 < C ? D[c + 1] : dr;
          const R hp = c >= 1 ? X[c - 1] : hl;
          if (KAHAN) kahan_add(D[c], cDv[KAHAN ? c : 0], (hp - X[c]) + cc * (du - D[c]));
          else D[c] = a * D[c] + (cc * du + (hp - X[c]));
          if (EDGE) D[c] = ((unsigned)(k0 + c) < (unsigned)nz) ? D[c] : (R)0;
        }
      }
    }
    if (damp) {   // absorbing layers: D^{n+1/2} at x = k
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const R g = absorb_factor<R>(I, (R)(k0 + c));
        D[c] *= g;
        if constexpr (KAHAN) cDv[c] *= g;
      }
    }
    if (tmask) tfsf_add(D, s, -1, 4, 2);   // one-way sources: D at node - 1 .. node

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

    // ---- D^{n+1/2} of every step, for the adjoint's segment recomputation
    if (A.dseg)
      store_cells<T, R, C>(A.dseg + (long long)(A.s0 + s + 1) * A.dseg_stride + I.off, k0, x0,
                           min(x0 + W, I.nz_pad), D);
  }

  const int hi = min(x0 + W, I.nz_pad);
  store_cells<T, R, C>(A.Bout + I.off, k0, x0, hi, B);
  store_cells<T, R, C>(A.Dout + I.off, k0, x0, hi, D);
}

// ------------------------------------------------ TMA bulk copies + mbarrier

// A bounded wait gives up after one second of device time (or kWaitLimit
// polls, a backstop that does not depend on the timer), far beyond any real
// tile copy.
constexpr long long kWaitLimit = 1LL << 24;
constexpr unsigned long long kWaitNs = 1000000000ull;
constexpr int kErrTimeout = 1;

__device__ __forceinline__ unsigned smem_u32(const void* p) {
  return static_cast<unsigned>(__cvta_generic_to_shared(p));
}
__device__ __forceinline__ void mbar_init(unsigned long long* bar, unsigned count) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void fence_proxy_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* bar, unsigned bytes) {
  asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
               : "memory");
}
// 1-D bulk copy global -> shared through the TMA unit; completion counts on `bar`.
__device__ __forceinline__ void bulk_g2s(void* dst, const void* src, unsigned bytes,
                                         unsigned long long* bar) {
  asm volatile(
      "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(
          smem_u32(dst)),
      "l"(src), "r"(bytes), "r"(smem_u32(bar))
      : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(unsigned long long* bar, unsigned phase) {
  unsigned ok;
  asm volatile(
      "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}"
      : "=r"(ok)
      : "r"(smem_u32(bar)), "r"(phase)
      : "memory");
  return ok != 0;
}
__device__ __forceinline__ unsigned long long global_ns() {
  unsigned long long t;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
  return t;
}
// Wait for phase `phase` of `bar`, giving up after kWaitNs of device time or
// kWaitLimit polls.
__device__ __forceinline__ bool mbar_wait_bounded(unsigned long long* bar, unsigned phase) {
  if (mbar_try_wait(bar, phase)) return true;
  const unsigned long long t0 = global_ns();
  for (long long it = 1; it < kWaitLimit; ++it) {
    if (mbar_try_wait(bar, phase)) return true;
    if ((it & 255) == 0 && global_ns() - t0 > kWaitNs) return false;
  }
  return false;
}

// Asynchronous 16-byte copy global -> shared (zero-filled when `valid` is false;
// the source address is then not read), and the waits on its groups.
__device__ __forceinline__ void cp_async16(void* sdst, const void* gsrc, bool valid) {
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;" ::"r"(smem_u32(sdst)), "l"(gsrc),
               "r"(valid ? 16 : 0)
               : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() { asm volatile("cp.async.wait_group %0;" ::"n"(N) : "memory"); }
// Wait until at most `pending` (0 .. 7) of this thread's copy groups are still in flight.
__device__ __forceinline__ void cp_async_wait_upto(int pending) {
  switch (pending) {
    case 0: cp_async_wait<0>(); break;
    case 1: cp_async_wait<1>(); break;
    case 2: cp_async_wait<2>(); break;
    case 3: cp_async_wait<3>(); break;
    case 4: cp_async_wait<4>(); break;
    case 5: cp_async_wait<5>(); break;
    case 6: cp_async_wait<6>(); break;
    default: cp_async_wait<7>(); break;
  }
}
// ------------------------------------------------ fast tile (common case)
//
// Moving perturbation, uniform mu, layered eps whose layers are wider than a
// lane's run (or uniform eps), tile away from the domain ends.  E' and H' are
// not formed: substituting them gives, with P_j = se_j D_j (level n-1/2),
//   v >= 0:  B'_j = (a + cb) B_j + c B_{j-1} - cb B_{j-2} + P_j - P_{j+1}
//            D'_k = a D_k + (c - cb) D_{k-1} + cb D_{k+1} + sm (B'_{k-1} - B'_k)
//   v <  0:  B'_j = (a - cb) B_j + c B_{j+1} + cb B_{j+2} + P_j - P_{j+1}
//            D'_k = a D_k + (c + cb) D_{k+1} - cb D_{k-1} + sm (B'_{k-1} - B'_k)
// (the same equations, regrouped).  Inside the tile B is carried as
// Bs = sm B (sm uniform), which removes the multiply by sm from the D update:
// Bs'_j = (same weights) Bs + sm (P_j - P_{j+1}) and D'_k = ... + Bs'_{k-1} - Bs'_k;
// the factor sm is applied to the layer values, so P holds sm se D.  The
// material of a lane is tracked with the two layer boundaries around its first
// cell k0: d = zq + dq h - k0 2^32 grows by 2 dq per step, and cells
// c >= ceil(d / 2^32) of the run lie beyond the boundary.  The B update takes
// one multiplier per lane (the layer of the whole run); the few lanes with a
// boundary inside their run then add the difference of the two layers' P.

struct BoundaryTrack {
  long long dprev, dnext;     // zq_b + dq h - k0 2^32 of the boundaries around k0
  long long dnext2;           // the boundary after dnext (tracked when a run can hold two)
  int bnext;                  // index of the next boundary (first with d > 0)
};

// Boundaries a lane's run of C cells may hold in the fast kernel: the wider
// runs track a second one, so layers need only be wider than C / 2.
__host__ __device__ constexpr int fast_boundaries_per_run(int C) { return C > 16 ? 2 : 1; }

constexpr long long FAR_AWAY = 1LL << 61;

__device__ __forceinline__ long long track_d(const long long* __restrict__ zq, int b, int nb,
                                             long long off) {
  if (b < 0) return -FAR_AWAY;
  if (b >= nb) return FAR_AWAY;
  return __ldg(zq + b) + off;
}

// B^n of a fast tile with P_c = vc(c) D_c (level n-1/2) for cell c of the
// lane's run; P of the next lane's cell 0 comes by shuffle.
// x, or zero when z (the argument is evaluated by every lane first).
template <typename R>
__device__ __forceinline__ R sel0(bool z, R x) { return z ? (R)0 : x; }

// zl / zr: the cells left of the run / right of it are outside the domain (zero).
template <int C, bool POS, typename R, typename VC>
__device__ __forceinline__ void fast_b_update_cells(R (&B)[C], const R (&D)[C], VC vc, R bB0, R cc, R cb,
                                                    bool zl = false, bool zr = false) {
  // every lane takes part in each shuffle; the ends of the domain are applied after
  const R pr = sel0(zr, __shfl_down_sync(FULL, vc(0) * D[0], 1));
  if (POS) {
    const R bl1 = sel0(zl, __shfl_up_sync(FULL, B[C - 1], 1));
    const R bl2 = sel0(zl, __shfl_up_sync(FULL, B[C - 2], 1));
    R pn = pr;
#pragma unroll
    for (int c = C - 1; c >= 0; --c) {
      const R b1 = c >= 1 ? B[c - 1] : bl1;
      const R b2 = c >= 2 ? B[c - 2] : (c == 1 ? bl1 : bl2);
      const R pc = vc(c) * D[c];
      B[c] = bB0 * B[c] + (cc * b1 + (-cb * b2 + (pc - pn)));
      pn = pc;
    }
  } else {
    const R br1 = sel0(zr, __shfl_down_sync(FULL, B[0], 1));
    const R br2 = sel0(zr, __shfl_down_sync(FULL, B[1], 1));
    R pc = vc(0) * D[0];
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const R b1 = c + 1 < C ? B[c + 1] : br1;
      const R b2 = c + 2 < C ? B[c + 2] : (c + 2 == C ? br1 : br2);
      const R pn = c + 1 < C ? vc(c + 1) * D[c + 1] : pr;
      B[c] = bB0 * B[c] + (cc * b1 + (cb * b2 + (pc - pn)));
      pc = pn;
    }
  }
}

// The same with one multiplier v for the whole run.
template <int C, bool POS, typename R>
__device__ __forceinline__ void fast_b_update(R (&B)[C], const R (&D)[C], R v, R bB0, R cc, R cb) {
  fast_b_update_cells<C, POS>(B, D, [v](int) { return v; }, bB0, cc, cb);
}

// D^{n+1/2} of a fast tile, in place, walking from the downwind end: the term
// of the next cell that needs this cell's old D (its downwind neighbour) is
// formed before that D is overwritten.  B is (S/mu) B^n.
template <int C, bool POS, typename R>
__device__ __forceinline__ void fast_d_update(const R (&B)[C], R (&D)[C], R a, R bD1, R bD2,
                                              bool zl = false, bool zr = false) {
  const R dl = sel0(zl, __shfl_up_sync(FULL, D[C - 1], 1));
  const R dr = sel0(zr, __shfl_down_sync(FULL, D[0], 1));
  const R bnl = sel0(zl, __shfl_up_sync(FULL, B[C - 1], 1));
  if (POS) {
    R part = bD2 * dr + (B[C - 2] - B[C - 1]);
#pragma unroll
    for (int c = C - 1; c >= 0; --c) {
      R next = 0;
      if (c >= 1) next = bD2 * D[c] + ((c >= 2 ? B[c - 2] : bnl) - B[c - 1]);
      const R left = c >= 1 ? D[c - 1] : dl;
      D[c] = a * D[c] + (bD1 * left + part);
      part = next;
    }
  } else {
    R part = bD2 * dl + (bnl - B[0]);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      R next = 0;
      if (c + 1 < C) next = bD2 * D[c] + (B[c] - B[c + 1]);
      const R right = c + 1 < C ? D[c + 1] : dr;
      D[c] = a * D[c] + (bD1 * right + part);
      part = next;
    }
  }
}

// sB, sD: the tile's 32 C cells of B and D, and sT: the tracker state saved
// for the tile by the previous launch (NULL: none kept), all in shared memory.
// refill() is called once every lane has read them: it may overwrite them.
// DAMP: the tile reaches an absorbing layer (a separate instantiation, so that
// the damping adds nothing to the loops of the other tiles).
template <int C, int TB, bool POS, typename T, bool DAMP, typename Refill>
__device__ __forceinline__ void run_tile_fast(const BlockArgs<T>& A, const InstDev& I, const FastTile& ft,
                                              long long n0, const T* sB, const T* sD,
                                              const TrackTile* sT, int t, Refill&& refill) {
  using R = typename Real<T>::type;
  using V2 = typename TabOf<R>::V;
  const int lane = threadIdx.x & 31;
  constexpr int L = tile_margin(TB, POS, 16 / sizeof(T));     // x0 - base
  constexpr int W = tile_width(C, TB, POS, 16 / sizeof(T));   // output cells
  const int x0 = ft.x0;
  const int base = ft.base;                        // x0 - L, or moved inside the domain at its ends
  const int k0 = base + lane * C;
  (void)L;

  R B[C], D[C];
  {
    constexpr int V = 16 / sizeof(T);
#pragma unroll
    for (int j = 0; j < C / V; ++j) {
      unpack(*reinterpret_cast<const uint4*>(sB + lane * C + j * V), &B[j * V], T());
      unpack(*reinterpret_cast<const uint4*>(sD + lane * C + j * V), &D[j * V], T());
    }
  }
  R sm;                                             // S / mu, uniform in a fast tile
  if constexpr (sizeof(R) == 4) sm = I.sm32;
  else sm = __ldg(&A.tb.tabH[I.tab].x);
#pragma unroll
  for (int c = 0; c < C; ++c) B[c] *= sm;          // Bs = sm B

  const R a = coef<R>(I.a, I.a32), cc = coef<R>(I.c, I.c32), cb = coef<R>(I.cb, I.cb32);
  const R bB0 = POS ? a + cb : a - cb;            // weight of B_j
  const R bD1 = POS ? cc - cb : cc + cb;          // weight of the upwind D neighbour
  const R bD2 = POS ? cb : -cb;                   // weight of the downwind D neighbour
  const V2* __restrict__ tv = TabOf<R>::get(A.tb, true) + I.tab;
  const long long* __restrict__ zq = A.tb.zq + I.tab;
  const int nb = I.n - 1;
  const long long dq2 = 2 * I.dq;

  // boundary tracker at half level h = 2 n0 + 1 (the first E' of this launch):
  // the state the previous launch left for this tile if it ended at n0, else
  // found by binary search.
  constexpr int NB = fast_boundaries_per_run(C);
  BoundaryTrack tr{};
  R vL, vM = 0, vR;      // sm se of the layers: k0's, past dnext (NB = 2: up to dnext2), past the last tracked
  auto load_layers = [&]() {
    vL = sm * __ldg(tv + tr.bnext).x;
    if constexpr (NB == 2) {
      vM = sm * __ldg(tv + min(tr.bnext + 1, nb)).x;
      vR = sm * __ldg(tv + min(tr.bnext + 2, nb)).x;
    } else {
      vR = sm * __ldg(tv + min(tr.bnext + 1, nb)).x;
    }
  };
  if (sT && sT->n == n0) {
    const TrackLane& s = sT->lane[lane];
    tr.dprev = s.dprev;
    tr.dnext = s.dnext;
    tr.dnext2 = s.dnext2;
    tr.bnext = s.bnext;
    if constexpr (sizeof(R) == 4) {
      vL = s.vL;
      vM = s.vM;
      vR = s.vR;
    } else {
      load_layers();
    }
  } else {
    const long long offh = I.dq * (2 * n0 + 1);
    const long long off0 = offh - ((long long)k0 << 32);
    tr.bnext = count_at_or_left(zq, nb, offh, k0);
    tr.dprev = track_d(zq, tr.bnext - 1, nb, off0);
    tr.dnext = track_d(zq, tr.bnext, nb, off0);
    tr.dnext2 = NB == 2 ? track_d(zq, tr.bnext + 1, nb, off0) : FAR_AWAY;
    load_layers();
  }
  __syncwarp();   // every lane has read its tile data: the buffer may be refilled
  refill();

  const unsigned smask = A.src_amp ? ft.smask : 0u;
  const unsigned pmask = A.record ? ft.pmask : 0u;

  // A quiet tile has no source or probe, and in no lane does a boundary pass
  // the lane's first cell or lie inside its run during this launch: every lane
  // then keeps one multiplier and only the stencil arithmetic remains.
  bool quiet;
  {
    const long long span = (long long)(A.nsteps - 1) * dq2;   // dnext moves by this over the launch
    const int c1a = (int)((tr.dnext + 0xFFFFFFFFLL) >> 32);          // first step
    const int c1b = (int)((tr.dnext + span + 0xFFFFFFFFLL) >> 32);   // last step
    const bool no_event = POS ? tr.dprev + span + dq2 <= 0 : tr.dnext + span + dq2 > 0;
    const bool one_side = POS ? (c1a >= C || c1b <= 0) : (c1a <= 0 || c1b >= C);
    quiet = !DAMP && __all_sync(FULL, (smask | pmask) == 0u && ft.edge == 0 && no_event && one_side);
  }
  if (quiet) {
    const int c1 = (int)((tr.dnext + 0xFFFFFFFFLL) >> 32);
    const R v = c1 <= 0 ? vR : vL;
    for (int s = 0; s < A.nsteps; ++s) {
      fast_b_update<C, POS>(B, D, v, bB0, cc, cb);
      fast_d_update<C, POS>(B, D, a, bD1, bD2);
    }
    tr.dprev += (long long)A.nsteps * dq2;
    tr.dnext += (long long)A.nsteps * dq2;
    if constexpr (NB == 2) tr.dnext2 += (long long)A.nsteps * dq2;
  } else {
  // Tiles at the ends of the domain (Sec. 4 reading: all fields are zero outside
  // [0, nz), with E*_nz = H*_-1 = 0): the neighbours beyond an end read as zero,
  // the cells of lane 31 at or past nz are held at zero, and the two terms where
  // the fused update differs from those boundary values are corrected:
  // H'_-1 = 0 adds cb D_0 to D_0, and for v >= 0 E'_nz = 0 subtracts
  // cb (B_nz-1 + B_nz-2) from B_nz-1.
  const bool ledge = (ft.edge & 1) != 0, redge = (ft.edge & 2) != 0;
  const bool zl = ledge && lane == 0, zr = redge && lane == 31;
  const int rpast = ft.edge >> 8;                  // cells of the window at or past nz (< 16 / sizeof(T))
  constexpr int VW = 16 / sizeof(T);
  auto zero_past_end = [&](R (&X)[C]) {
#pragma unroll
    for (int c = C - VW + 1; c < C; ++c)
      if (zr && c >= C - rpast) X[c] = (R)0;
  };
  if (redge) {
    zero_past_end(B);
    zero_past_end(D);
  }
  // absorbing layers: each sample is multiplied after its update (x = k for D,
  // k + 1/2 for B; B is carried as (S/mu) B, which the factor leaves
  // proportional).  The layer's parameters are re-read from the instance
  // record in global memory at each use, so no register stays reserved for them.
  const InstDev* __restrict__ gI = A.inst + ft.inst;
  auto damp_cells = [gI, k0](R (&X)[C], R half) {
    const R aw = (R)__ldg(&gI->abs_w), aright = (R)(__ldg(&gI->nz) - 1) - aw, ainv = (R)1 / aw;
    const R asig = (R)__ldg(&gI->abs_sigma);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const R x = (R)(k0 + c) + half;
      const R d = x < aw ? (aw - x) * ainv : (x > aright ? (x - aright) * ainv : (R)0);
      X[c] *= exp(-asig * d * d);
    }
  };
  for (int s = 0; s < A.nsteps; ++s) {
    // ---- material at level n-1/2 for this lane's cells: c >= c1 lies beyond the next boundary
    const int c1 = (int)((tr.dnext + 0xFFFFFFFFLL) >> 32);

    R bend = 0;                          // right end, v >= 0: B_nz-1 + B_nz-2 at level n-1
    if (POS && redge) {
#pragma unroll
      for (int q = 0; q < VW; ++q)
        if (rpast == q) bend = B[C - 1 - q] + B[C - 2 - q];
    }

    // ---- B^n with P_c = v_c D_c: cells c >= c1 take vM (NB = 2) or vR, c >= c2 vR.
    // Wide runs keep one copy of the update (per-cell multiplier) so that the
    // loop fits the instruction cache next to the quiet loop; 16-cell runs
    // also keep a copy with one multiplier for warps without a boundary inside.
    if constexpr (NB == 2) {
      const int c2 = (int)((tr.dnext2 + 0xFFFFFFFFLL) >> 32);
      fast_b_update_cells<C, POS>(B, D, [&](int c) { return c >= c2 ? vR : (c >= c1 ? vM : vL); },
                                  bB0, cc, cb, zl, zr);
    } else {
      if (__any_sync(FULL, c1 < C))
        fast_b_update_cells<C, POS>(B, D, [&](int c) { return c >= c1 ? vR : vL; }, bB0, cc, cb, zl, zr);
      else
        fast_b_update_cells<C, POS>(B, D, [&](int) { return vL; }, bB0, cc, cb, zl, zr);
    }
    if (redge) {
      if (POS) {
#pragma unroll
        for (int q = 0; q < VW; ++q)
          if (zr && rpast == q) B[C - 1 - q] -= cb * bend;
      }
      zero_past_end(B);
    }
    if constexpr (DAMP) damp_cells(B, (R)0.5);
    const R d0 = D[0];                   // left end: D_0 at level n-1/2

    // ---- D^{n+1/2}
    fast_d_update<C, POS>(B, D, a, bD1, bD2, zl, zr);
    if (ledge && zl) D[0] += cb * d0;
    if (redge) zero_past_end(D);
    if constexpr (DAMP) damp_cells(D, (R)0);

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

    // ---- advance the boundary tracker to level n+1/2.  With v >= 0 the d
    // values only grow, so only the previous boundary can pass k0; with
    // v < 0 only the next one can.
    tr.dprev += dq2;
    tr.dnext += dq2;
    if constexpr (NB == 2) tr.dnext2 += dq2;
    if (POS && tr.dprev > 0) {            // the previous boundary moved past k0
      if constexpr (NB == 2) tr.dnext2 = tr.dnext;
      tr.dnext = tr.dprev;
      tr.bnext -= 1;
      const long long offn = I.dq * (2 * (n0 + s + 1) + 1) - ((long long)k0 << 32);
      tr.dprev = track_d(zq, tr.bnext - 1, nb, offn);
      load_layers();
    } else if (!POS && tr.dnext <= 0) {   // the next boundary moved to or behind k0
      tr.dprev = tr.dnext;
      tr.bnext += 1;
      const long long offn = I.dq * (2 * (n0 + s + 1) + 1) - ((long long)k0 << 32);
      if constexpr (NB == 2) {
        tr.dnext = tr.dnext2;
        tr.dnext2 = track_d(zq, tr.bnext + 1, nb, offn);
      } else {
        tr.dnext = track_d(zq, tr.bnext, nb, offn);
      }
      load_layers();
    }

    // ---- probes: E = D / eps at level n+1/2
    for (unsigned m = pmask; m; m &= m - 1) {
      const int q = __ffs(m) - 1;
      const int node = A.prbs[I.prb0 + q].node;
      const int rel = node - base;
      if (lane == rel / C) {
        R sep, cbp;
        node_coef<false, true>(I, A.tb, I.dq * (2 * (n0 + s + 1) + 1), node, sep, cbp);
        A.samples[(long long)(I.prb0 + q) * A.chunk_stride + A.s0 + s] =
            (double)(pick(D, rel % C) * sep * (R)I.inv_S);
      }
    }
  }
  }

  if (A.track) {
    TrackLane o;
    o.dprev = tr.dprev;
    o.dnext = tr.dnext;
    o.dnext2 = tr.dnext2;
    o.vL = (float)vL;
    o.vM = (float)vM;
    o.vR = (float)vR;
    o.bnext = tr.bnext;
    o.pad = 0;
    A.track[t].lane[lane] = o;
    if (lane == 0) A.track[t].n = n0 + A.nsteps;
  }
  // back to B.  A plain multiplication by the rounded 1/sm would scale B by
  // the same factor sm fl(1/sm) = 1 - e at every launch; the residual e,
  // exact in one FMA, corrects that (a division per cell would be exact too,
  // but costs a quarter of the kernel's time on the crystal).
  {
    const R r = (R)1 / sm;
    const R e = fma(-sm, r, (R)1);
#pragma unroll
    for (int c = 0; c < C; ++c) {
      const R p = B[c] * r;
      B[c] = fma(p, e, p);
    }
  }
  const int hi = min(x0 + W, I.nz_pad);
  store_cells<T, R, C>(A.Bout + I.off, k0, x0, hi, B);
  store_cells<T, R, C>(A.Dout + I.off, k0, x0, hi, D);
}

// Blocks per SM the general kernel's registers are held to: runs of up to 8
// cells in FP32 arithmetic fit in fewer registers, and the batches that
// choose them are small (few warps), so occupancy pays there; wider runs,
// FP64 arithmetic and the compensated tier keep the compiler's choice (0: no
// bound).
__host__ __device__ constexpr int general_min_blocks(int C, int real_bytes, bool kahan) {
  return (kahan || real_bytes != 4) ? 0 : (C <= 4 ? 6 : (C <= 8 ? 4 : 0));
}

template <int C, int TB, bool MATTER, typename T, bool KAHAN = false>
__global__ void __launch_bounds__(128, general_min_blocks(C, sizeof(typename Real<T>::type), KAHAN)) block_kernel(const BlockArgs<T> A) {
  const int warps_per_block = blockDim.x >> 5;
  const int gw = blockIdx.x * warps_per_block + (threadIdx.x >> 5);
  const int nw = gridDim.x * warps_per_block;
  const long long n0 = *A.n_done + A.s0;
  const int nt = A.queue ? *(volatile int*)A.qcount : A.n_tiles;
  for (int i = gw; i < nt; i += nw) {
    const int t = A.queue ? A.queue[i] : i;
    const int2 tl = A.tiles[t];
    const InstDev I = A.inst[tl.x];
    const int x0 = tl.y;
    constexpr int V = 16 / sizeof(T);
    if (I.flags & F_POS) {
      constexpr int W = tile_width(C, TB, true, V);
      const int base = x0 - tile_margin(TB, true, V);
      if (base < 0 || base + 32 * C > I.nz) run_tile<C, TB, true, MATTER, true, T, KAHAN>(A, I, x0, W, n0);
      else run_tile<C, TB, true, MATTER, false, T, KAHAN>(A, I, x0, W, n0);
    } else {
      constexpr int W = tile_width(C, TB, false, V);
      const int base = x0 - tile_margin(TB, false, V);
      if (base < 0 || base + 32 * C > I.nz) run_tile<C, TB, false, MATTER, true, T, KAHAN>(A, I, x0, W, n0);
      else run_tile<C, TB, false, MATTER, false, T, KAHAN>(A, I, x0, W, n0);
    }
  }
  if (A.queue) {
    // the last block out empties the queue for the next launch (every warp has read
    // its length by then)
    __syncthreads();
    if (threadIdx.x == 0 && atomicAdd(A.qcount + 1, 1) == (int)gridDim.x - 1) {
      atomicExch(A.qcount, 0);
      atomicExch(A.qcount + 1, 0);
    }
  }
}

// ------------------------------------------------ uniform tiles of the general lists
//
// A tile of the general lists whose window lies inside the domain, sees one ε
// value and one μ value over the whole launch (uniform_sides) and holds no
// absorbing layer, no recorded probe and no one-way source's correction cells
// steps in uniform_kernel with E' and H' substituted, the regrouping of the
// fast kernel here with the couplings cbe, cbh of the two uniform values (for
// moving perturbation both are cb):
//   v >= 0:  B'_j = (a + cbe) B_j + c B_{j-1} - cbe B_{j-2} + se (D_j - D_{j+1})
//            D'_k = a D_k + (c - cbh) D_{k-1} + cbh D_{k+1} + sm (B'_{k-1} - B'_k)
//   v <  0:  B'_j = (a - cbe) B_j + c B_{j+1} + cbe B_{j+2} + se (D_j - D_{j+1})
//            D'_k = a D_k + (c + cbh) D_{k+1} - cbh D_{k-1} + sm (B'_{k-1} - B'_k)
// (with the FP32 weights of reading R16 the sums a + cbe, c - cbh, ... are
// exact).  It appends every other tile to the queue that block_kernel then
// takes, so the general kernel's registers and code serve only the tiles that
// need them.  Returns whether the tile was stepped.
// `pre`: the window's B and D (32 C elements each), already copied into shared memory;
// `refill` is called once on every path, as soon as `pre` has been read or is not needed.
template <int C, int TB, bool POS, typename T, typename Refill>
__device__ __forceinline__ bool run_tile_uniform(const BlockArgs<T>& A, const InstDev& I, int x0, int W,
                                                 long long n0, const T* pre, Refill&& refill) {
  using R = typename Real<T>::type;
  const int lane = threadIdx.x & 31;
  constexpr int L = tile_margin(TB, POS, 16 / sizeof(T));
  constexpr int SPAN = 32 * C;
  const int base = x0 - L;
  bool take = !(base < 0 || base + SPAN > I.nz || window_absorbs(I, base, SPAN));
  if (take && A.record)
    for (int q = 0; q < I.nprb; ++q) {
      const int node = A.prbs[I.prb0 + q].node;
      if (node >= x0 && node < x0 + W) take = false;
    }
  if (take && A.n_tfsf > 0)
    for (int q = 0; q < I.ntf; ++q) {
      const int node = A.tfsf[I.tf0 + q].node;
      if (node + 1 >= base && node - 2 < base + SPAN) take = false;
    }
  bool eps_const = false, mu_const = false;
  int rE = 0, rH = 0;
  if (take) {
    uniform_sides(I, A.tb, base, SPAN, n0, A.nsteps, eps_const, mu_const, rE, rH);
    take = eps_const && mu_const;
  }
  if (!take) {
    refill();
    return false;
  }

  const bool lin = (I.flags & F_LINEAR) != 0, matter = (I.flags & F_MATTER) != 0;
  const auto e0 = __ldg(TabOf<R>::get(A.tb, true) + I.tab + rE);
  const auto h0 = __ldg(TabOf<R>::get(A.tb, false) + I.tab + rH);
  // (uniform values: LINEAR tables hold raw (eps, mu), LAYERS tables the coefficients)
  const R se = lin ? (R)I.S / e0.x : e0.x, sm = lin ? (R)I.S / h0.y : h0.x;
  const R cb = coef<R>(I.cb, I.cb32);
  const R cbe = matter ? (R)e0.y : cb, cbh = matter ? (R)h0.y : cb;
  const R a = coef<R>(I.a, I.a32), cc = coef<R>(I.c, I.c32);
  const R kb0 = POS ? a + cbe : a - cbe;     // B_j
  const R kb2 = POS ? -cbe : cbe;            // B_{j-2} (v >= 0) or B_{j+2} (v < 0)
  const R kdu = POS ? cc - cbh : cc + cbh;   // upwind D neighbour
  const R kdd = POS ? cbh : -cbh;            // downwind D neighbour
  const int k0 = base + lane * C;

  unsigned smask = 0;
  if (A.src_amp)
    for (int q = 0; q < I.nsrc && q < 32; ++q) {
      const int node = A.srcs[I.src0 + q].node;
      if (node >= base && node < base + SPAN) smask |= 1u << q;
    }

  R B[C], D[C];
  {
    constexpr int V = 16 / sizeof(T);
#pragma unroll
    for (int j = 0; j < C / V; ++j) {
      unpack(*reinterpret_cast<const uint4*>(pre + lane * C + j * V), &B[j * V], T());
      unpack(*reinterpret_cast<const uint4*>(pre + SPAN + lane * C + j * V), &D[j * V], T());
    }
  }
  refill();
  for (int s = 0; s < A.nsteps; ++s) {
    // ---- B^n
    const R dr = __shfl_down_sync(FULL, D[0], 1);
    if (POS) {
      const R bl1 = __shfl_up_sync(FULL, B[C - 1], 1), bl2 = __shfl_up_sync(FULL, B[C - 2], 1);
#pragma unroll
      for (int c = C - 1; c >= 0; --c) {
        const R b1 = c >= 1 ? B[c - 1] : bl1;
        const R b2 = c >= 2 ? B[c - 2] : (c == 1 ? bl1 : bl2);
        const R d1 = c + 1 < C ? D[c + 1] : dr;
        B[c] = kb0 * B[c] + (cc * b1 + (kb2 * b2 + se * (D[c] - d1)));
      }
    } else {
      const R br1 = __shfl_down_sync(FULL, B[0], 1), br2 = __shfl_down_sync(FULL, B[1], 1);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const R b1 = c + 1 < C ? B[c + 1] : br1;
        const R b2 = c + 2 < C ? B[c + 2] : (c + 2 == C ? br1 : br2);
        const R d1 = c + 1 < C ? D[c + 1] : dr;
        B[c] = kb0 * B[c] + (cc * b1 + (kb2 * b2 + se * (D[c] - d1)));
      }
    }
    // ---- D^{n+1/2}
    {
      const R bl = __shfl_up_sync(FULL, B[C - 1], 1), dl = __shfl_up_sync(FULL, D[C - 1], 1);
      R Dn[C];
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const R dm = c >= 1 ? D[c - 1] : dl, dp = c + 1 < C ? D[c + 1] : dr;
        const R bm = c >= 1 ? B[c - 1] : bl;
        Dn[c] = a * D[c] + ((POS ? kdu * dm + kdd * dp : kdu * dp + kdd * dm) + sm * (bm - B[c]));
      }
#pragma unroll
      for (int c = 0; c < C; ++c) D[c] = Dn[c];
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
    // ---- D^{n+1/2} of every step, for the adjoint's segment recomputation
    if (A.dseg)
      store_cells<T, R, C>(A.dseg + (long long)(A.s0 + s + 1) * A.dseg_stride + I.off, k0, x0, x0 + W, D);
  }
  store_cells<T, R, C>(A.Bout + I.off, k0, x0, x0 + W, B);
  store_cells<T, R, C>(A.Dout + I.off, k0, x0, x0 + W, D);
  return true;
}

// Blocks per SM the uniform kernel's registers are held to.
__host__ __device__ constexpr int uniform_min_blocks(int C, int real_bytes) {
  return real_bytes != 4 ? 0 : (C <= 8 ? 8 : (C <= 16 ? 6 : 4));
}

template <int C, int TB, typename T>
__global__ void __launch_bounds__(128, uniform_min_blocks(C, sizeof(typename Real<T>::type)))
    uniform_kernel(const BlockArgs<T> A) {
  constexpr int V = 16 / sizeof(T), SPAN = 32 * C;
  // per warp: the window's B and D of the tile being stepped, copied asynchronously while
  // the warp steps the tile before it (each lane copies and reads only its own cells)
  __shared__ __align__(16) T ubuf[4][2 * SPAN];
  const int wib = __shfl_sync(FULL, (int)(threadIdx.x >> 5), 0), lane = threadIdx.x & 31;
  const int gw = blockIdx.x * 4 + wib, nw = gridDim.x * 4;
  const long long n0 = *A.n_done + A.s0;
  T* buf = ubuf[wib];
  auto prefetch = [&](int t) {
    if (t >= A.n_tiles) return;
    const int2 tl = A.tiles[t];
    const InstDev& J = A.inst[tl.x];
    const int base = tl.y - ((J.flags & F_POS) ? tile_margin(TB, true, V) : tile_margin(TB, false, V));
#pragma unroll
    for (int j = 0; j < C / V; ++j) {
      const int kc = base + lane * C + j * V;
      const bool ok = kc >= 0 && kc < J.nz_pad;
      const long long e = J.off + (ok ? kc : 0);
      cp_async16(buf + lane * C + j * V, A.Bin + e, ok);
      cp_async16(buf + SPAN + lane * C + j * V, A.Din + e, ok);
    }
    cp_async_commit();
  };
  prefetch(gw);
  for (int t = gw; t < A.n_tiles; t += nw) {
    const int2 tl = A.tiles[t];
    const InstDev I = A.inst[tl.x];
    cp_async_wait<0>();
    auto refill = [&]() { prefetch(t + nw); };
    const bool done = (I.flags & F_POS)
                          ? run_tile_uniform<C, TB, true, T>(A, I, tl.y, tile_width(C, TB, true, V), n0, buf, refill)
                          : run_tile_uniform<C, TB, false, T>(A, I, tl.y, tile_width(C, TB, false, V), n0, buf,
                                                              refill);
    if (!done && lane == 0) A.queue[atomicAdd(A.qcount, 1)] = t;
  }
}

// Interior tiles of moving-perturbation instances with uniform mu and wide
// (or no) layers; the host sorts such tiles into their own list.  Each warp
// walks its tiles with one shared-memory buffer: as soon as the lanes hold a
// tile's cells in registers, bulk copies start bringing the next tile's
// cells, instance record, tile record and saved tracker state into it, and
// they land while the warp steps the current tile.
template <int C, int TB, typename T, int MB, bool DAMP = false>
__global__ void __launch_bounds__(128, MB) fast_kernel(const BlockArgs<T> A) {
  constexpr int WPB = 4;                    // warps per block (blockDim.x == 128)
  constexpr int CELLS = 32 * C;
  constexpr unsigned BYTES = CELLS * sizeof(T);
  __shared__ __align__(128) T sbuf[WPB][2][CELLS];      // [warp][B, D][cell]
  __shared__ __align__(16) InstDev sinst[WPB];
  __shared__ __align__(16) FastTile sft[WPB];
  __shared__ __align__(16) TrackTile strk[WPB];
  __shared__ __align__(8) unsigned long long sbar[WPB];
  // (the warp index taken by shuffle is known to the compiler to be warp-uniform,
  // which lets it keep the tile bookkeeping out of the per-lane registers)
  const int wib = __shfl_sync(0xffffffffu, (int)(threadIdx.x >> 5), 0), lane = threadIdx.x & 31;
  const int gw = blockIdx.x * WPB + wib;
  const int nw = gridDim.x * WPB;
  const long long n0 = *A.n_done + A.s0;
  const unsigned tx = 2 * BYTES + (unsigned)sizeof(InstDev) + (unsigned)sizeof(FastTile) +
                      (A.track ? (unsigned)sizeof(TrackTile) : 0u);
  if (lane == 0) {
    mbar_init(&sbar[wib], 1);
    fence_mbar_init();
  }
  __syncwarp();

  // lane 0: input offset and instance of the tile to be prefetched next; the
  // record is read one tile ahead so that it is in registers when needed
  long long fe = 0;
  int fi = 0;
  auto fetch_record = [&](int t) {
    if (lane == 0 && t < A.n_tiles) {
      fe = A.ftiles[t].e;
      fi = A.ftiles[t].inst;
    }
  };
  // lane 0 starts the bulk copies of tile t into the warp's buffer
  auto prefetch = [&](int t) {
    if (lane == 0 && t < A.n_tiles) {
      fence_proxy_async();
      mbar_expect_tx(&sbar[wib], tx);
      if (A.stall) return;   // test hook: no copy is started, so the wait for it runs out
      bulk_g2s(&sbuf[wib][0][0], A.Bin + fe, BYTES, &sbar[wib]);
      bulk_g2s(&sbuf[wib][1][0], A.Din + fe, BYTES, &sbar[wib]);
      bulk_g2s(&sinst[wib], A.inst + fi, sizeof(InstDev), &sbar[wib]);
      bulk_g2s(&sft[wib], A.ftiles + t, sizeof(FastTile), &sbar[wib]);
      if (A.track) bulk_g2s(&strk[wib], A.track + t, sizeof(TrackTile), &sbar[wib]);
    }
  };

  unsigned phase = 0u;
  fetch_record(gw);
  prefetch(gw);
  fetch_record(gw + nw);
  for (int t = gw; t < A.n_tiles; t += nw) {
    const int tn = t + nw;
    const bool ok = __all_sync(FULL, mbar_wait_bounded(&sbar[wib], phase));
    if (!ok) {
      // give up: report, wait (bounded) for this warp's copies still in flight, leave
      if (lane == 0) atomicOr(A.err, kErrTimeout);
      mbar_wait_bounded(&sbar[wib], phase);
      return;
    }
    phase ^= 1u;
    const InstDev I = sinst[wib];
    const FastTile ft = sft[wib];
    const TrackTile* sT = A.track ? &strk[wib] : nullptr;
    auto refill = [&]() {
      prefetch(tn);
      fetch_record(tn + nw);
    };
    if (I.flags & F_POS)
      run_tile_fast<C, TB, true, T, DAMP>(A, I, ft, n0, sbuf[wib][0], sbuf[wib][1], sT, t, refill);
    else
      run_tile_fast<C, TB, false, T, DAMP>(A, I, ft, n0, sbuf[wib][0], sbuf[wib][1], sT, t, refill);
  }
}

// MB: blocks of 128 threads per SM the fast kernel is register-limited to.
template <int C, int TB, typename T, bool KAHAN = false, int MB = 4>
int launch_block_shape(int variant, const void* args, int grid, int block, cudaStream_t st) {
  const BlockArgs<T>& a = *static_cast<const BlockArgs<T>*>(args);
  if (variant == 2 && !KAHAN) fast_kernel<C, TB, T, MB><<<grid, block, 0, st>>>(a);
  else if (variant == 3 && !KAHAN) fast_kernel<C, TB, T, MB, true><<<grid, block, 0, st>>>(a);
  else if (variant == 4 && !KAHAN) uniform_kernel<C, TB, T><<<grid, block, 0, st>>>(a);
  else if (variant == 1) block_kernel<C, TB, true, T, KAHAN><<<grid, block, 0, st>>>(a);
  else if (variant == 0) block_kernel<C, TB, false, T, KAHAN><<<grid, block, 0, st>>>(a);
  else return (int)cudaErrorInvalidValue;
  return (int)cudaGetLastError();
}

template <int C, int TB, typename T, bool KAHAN = false, int MB = 4>
int occupancy_block_shape(int variant, int block, int* nb) {
  if (variant == 2 && !KAHAN) {
    // MB blocks of the fast kernel need MB x its static shared memory: ask for the largest carveout
    const cudaError_t e = cudaFuncSetAttribute(fast_kernel<C, TB, T, MB>,
                                               cudaFuncAttributePreferredSharedMemoryCarveout,
                                               (int)cudaSharedmemCarveoutMaxShared);
    if (e != cudaSuccess) return (int)e;
    const cudaError_t e3 = cudaFuncSetAttribute(fast_kernel<C, TB, T, MB, true>,
                                                cudaFuncAttributePreferredSharedMemoryCarveout,
                                                (int)cudaSharedmemCarveoutMaxShared);
    if (e3 != cudaSuccess) return (int)e3;
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, fast_kernel<C, TB, T, MB>, block, 0);
  }
  if (variant == 4 && !KAHAN)
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, uniform_kernel<C, TB, T>, block, 0);
  if (variant == 1)
    return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, block_kernel<C, TB, true, T, KAHAN>,
                                                              block, 0);
  return (int)cudaOccupancyMaxActiveBlocksPerMultiprocessor(nb, block_kernel<C, TB, false, T, KAHAN>,
                                                            block, 0);
}

// Whether an instance's interior tiles can take the fast path for C cells per lane.
__host__ __device__ inline bool fast_eligible(const InstDev& I, int C) {
  // layers wider than C cells (C / 2 when the kernel tracks two boundaries per run)
  const bool wide = fast_boundaries_per_run(C) == 2 ? 2 * I.minw > C : I.minw > C;
  return !(I.flags & F_MATTER) && (I.flags & F_MU_CONST) && !(I.flags & F_LINEAR) &&
         ((I.flags & F_EPS_CONST) || wide);
}

}  // namespace gfdtd
