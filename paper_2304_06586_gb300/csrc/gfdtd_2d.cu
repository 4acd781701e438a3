// gfdtd_2d.cu -- the 2D TE generalized scheme (oblique incidence, slanted
// moving layers): kernels and the gfdtd2d_* entry points of include/gfdtd.h.
//
// Sec. 3 and Sec. 4 before the 1D reduction, for moving perturbation in the
// x-z plane (d/dy = 0), motion along z, E = E_y y^, B = (B_x, 0, B_z),
// D = D_y y^.  Eq. star and Eq. const_3d give E*_y = D_y/eps + v B_x,
// H*_x = B_x/mu + v D_y, H*_z = B_z/mu (v x B = v B_x y^, v x D = -v D_y x^;
// for E along y the star fields are tangential to any boundary in the x-z
// plane, Eq. EHstar_comp); Eq. Maxwell_star with curl(v x F) = -v dF/dz gives,
// with E' = S E*, H' = S H* and a = 1 - |v| S, c = |v| S, cb = S v / 2:
//   E'_{i,k}   = se D_{i,k} + cb (B_x,k-1 + B_x,k-2)            (v < 0: B_x,k + B_x,k+1)
//   B_x,i,k'   = a B_x + c B_x,k-1 + (E'_{i,k+1} - E'_{i,k})     (v < 0: c B_x,k+1)
//   B_z,i,k'   = a B_z + c B_z,k-1 - (E'_{i+1,k} - E'_{i,k}) / dx
//   H'x_{i,k}  = smx B_x,i,k + cb (D_k + D_k+1),  H'z_{i,k} = smz B_z,i,k
//   D_{i,k}'   = a D + c D_k-1 + (H'x_k - H'x_k-1) - (H'z_{i,k} - H'z_{i-1,k}) / dx
// (dz = 1, S = dt/dz; B_x at (i, k+1/2), B_z at (i+1/2, k), D at (i, k); x
// periodic over nx columns, every field zero beyond the z ends).  Along z this
// is the 1D update with b = -B_x; along x the plain Yee differences.
//
// GPU layout: one CTA per z-tile holds every column of the grid (nx <= 32, one
// warp per column, the lanes of a warp along z with C cells each in registers,
// as in the 1D kernel) and advances the tile TB steps; the neighbour columns'
// E' and H'z pass through shared memory (two block barriers per step).  The
// z-window of a tile is widened by the 1D dependency cone; x needs no halo
// because the CTA holds the whole periodic extent.
#include "../../include/gfdtd.h"
#include "gfdtd_block.cuh"
#include "gfdtd_medium.h"

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <string>
#include <vector>

namespace gfdtd {

constexpr int kMaxCols2D = 32;

template <typename T>
struct Args2D {
  const InstDev* inst;
  Tables tb;
  int nx;                  // columns (= warps of a CTA)
  long long stride;        // elements between columns (nz rounded up to a multiple of 32)
  double inv_dx;           // 1 / dx
  const long long* sx;     // per column i: the slant at x_i and at x_{i+1/2}, round(x slope 2^32)
  const T* Bx_in;
  const T* Bz_in;
  const T* D_in;
  T* Bx_out;
  T* Bz_out;
  T* D_out;
  const int* tiles;        // first output cell (z) of every tile
  int n_tiles;
  const SrcDev* srcs;      // line sources: node = z node
  const double* src_cos;   // cos(kx x_i) of source q at column i: src_cos[q nx + i]
  int nsrc;
  const double* src_amp;   // [source][step in chunk]
  const int2* prb;         // probes: (column, z node)
  int nprb;
  double* samples;         // [probe][step in chunk]
  int chunk_stride;
  const long long* n_done;
  int s0, nsteps;
};

// A lane's C consecutive values to and from shared memory in 16-byte pieces
// (C x sizeof(R) is a multiple of 16 and the row starts are 16-byte aligned).
template <int C, typename R>
__device__ __forceinline__ void st_run(R* p, const R (&x)[C]) {
  constexpr int V = 16 / sizeof(R);
#pragma unroll
  for (int j = 0; j < C; j += V) {
    if constexpr (V == 4) *reinterpret_cast<float4*>(p + j) = make_float4(x[j], x[j + 1], x[j + 2], x[j + 3]);
    else *reinterpret_cast<double2*>(p + j) = make_double2(x[j], x[j + 1]);
  }
}
template <int C, typename R>
__device__ __forceinline__ void ld_run(const R* p, R (&x)[C]) {
  constexpr int V = 16 / sizeof(R);
#pragma unroll
  for (int j = 0; j < C; j += V) {
    if constexpr (V == 4) {
      const float4 v = *reinterpret_cast<const float4*>(p + j);
      x[j] = v.x; x[j + 1] = v.y; x[j + 2] = v.z; x[j + 3] = v.w;
    } else {
      const double2 v = *reinterpret_cast<const double2*>(p + j);
      x[j] = v.x; x[j + 1] = v.y;
    }
  }
}

// One z-tile of every column.  EDGE: the window reaches a z end of the domain,
// so cells outside [0, nz) are held at zero after each update.
template <int C, int TB, bool POS, typename T, bool EDGE>
__device__ __forceinline__ void te2d_tile(const Args2D<T>& A, const InstDev& I, int x0,
                                          typename Real<T>::type* sE, typename Real<T>::type* sH) {
  using R = typename Real<T>::type;
  constexpr int V = 16 / sizeof(T);
  constexpr int L = tile_margin(TB, POS, V);
  constexpr int W = tile_width(C, TB, POS, V);
  constexpr int CELLS = 32 * C;
  const int col = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int colR = col + 1 == A.nx ? 0 : col + 1, colL = col == 0 ? A.nx - 1 : col - 1;
  const int nz = I.nz;
  const int base = x0 - L;
  const int k0 = base + lane * C;
  const long long row = (long long)col * A.stride;

  R Bx[C], Bz[C], D[C], X[C], hz[C];
  load_cells<T, R, C>(A.Bx_in + row, k0, (int)A.stride, Bx);
  load_cells<T, R, C>(A.Bz_in + row, k0, (int)A.stride, Bz);
  load_cells<T, R, C>(A.D_in + row, k0, (int)A.stride, D);

  const R a = coef<R>(I.a, I.a32), cc = coef<R>(I.c, I.c32), cb = coef<R>(I.cb, I.cb32);
  const R rdx = (R)A.inv_dx;
  // the slant: a node at x samples the profile shifted by round(x slope 2^32)
  const long long sxE = A.sx[2 * col], sxZ = A.sx[2 * col + 1];
  const bool eps_const = (I.flags & F_EPS_CONST) != 0, mu_const = (I.flags & F_MU_CONST) != 0;
  const auto e0 = __ldg(TabOf<R>::get(A.tb, true) + I.tab);
  const auto h0 = __ldg(TabOf<R>::get(A.tb, false) + I.tab);
  const long long n0 = *A.n_done + A.s0;
  const long long dq = I.dq;
  int liE = 0, liX = 0, liZ = 0;
  if (!eps_const || !mu_const) {
    liE = count_at_or_left(A.tb.zq + I.tab, I.n - 1, dq * (2 * n0 + 1) + sxE, k0);
    liX = count_at_or_left(A.tb.zq + I.tab, I.n - 1, dq * (2 * n0 + 2) - HALF_CELL + sxE, k0);
    liZ = count_at_or_left(A.tb.zq + I.tab, I.n - 1, dq * (2 * n0 + 2) + sxZ, k0);
  }
  auto inside = [&](int c) { return !EDGE || (unsigned)(k0 + c) < (unsigned)nz; };
  // the line sources in the window and this column's probes in the output range (bit masks)
  unsigned smask = 0, pmask = 0;
  for (int q = 0; q < A.nsrc && q < 32; ++q) {
    const int rel = A.srcs[q].node - base;
    if (rel >= 0 && rel < CELLS) smask |= 1u << q;
  }
  for (int q = 0; q < A.nprb && q < 32; ++q) {
    const int2 p = A.prb[q];
    if (p.x == col && p.y >= x0 && p.y < x0 + W) pmask |= 1u << q;
  }

  for (int s = 0; s < A.nsteps; ++s) {
    const long long n = n0 + s + 1;   // B^{n-1} -> B^n, D^{n-1/2} -> D^{n+1/2}

    // ---- E'^{n-1/2} = se D + cb Bsum (B_x at level n-1), into registers and shared memory
    {
      const R bl1 = __shfl_up_sync(FULL, Bx[C - 1], 1), bl2 = __shfl_up_sync(FULL, Bx[C - 2], 1);
      const R br1 = __shfl_down_sync(FULL, Bx[0], 1);
      auto upd = [&](int c, R se, R) {
        R bs;
        if (POS) {
          const R b1 = c >= 1 ? Bx[c - 1] : bl1;
          const R b2 = c >= 2 ? Bx[c - 2] : (c == 1 ? bl1 : bl2);
          bs = b1 + b2;
        } else {
          bs = Bx[c] + (c + 1 < C ? Bx[c + 1] : br1);
        }
        X[c] = inside(c) ? se * D[c] + cb * bs : (R)0;
      };
      if (!eps_const) {
        lane_apply<C, false, true, R>(I, A.tb, dq * (2 * n - 1) + sxE, k0, liE, upd);
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) upd(c, (R)e0.x, (R)0);
      }
      st_run<C, R>(sE + col * CELLS + lane * C, X);
    }
    __syncthreads();

    // ---- B_x^n, B_z^n (upwind differences at level n-1)
    {
      const R er = __shfl_down_sync(FULL, X[0], 1);
      const R bxl = __shfl_up_sync(FULL, Bx[C - 1], 1), bxr = __shfl_down_sync(FULL, Bx[0], 1);
      const R bzl = __shfl_up_sync(FULL, Bz[C - 1], 1), bzr = __shfl_down_sync(FULL, Bz[0], 1);
      R eR[C];
      ld_run<C, R>(sE + colR * CELLS + lane * C, eR);
      if (POS) {
#pragma unroll
        for (int c = C - 1; c >= 0; --c) {
          const R en = c + 1 < C ? X[c + 1] : er;
          const R bxu = c >= 1 ? Bx[c - 1] : bxl;
          const R bzu = c >= 1 ? Bz[c - 1] : bzl;
          Bx[c] = a * Bx[c] + (cc * bxu + (en - X[c]));
          Bz[c] = a * Bz[c] + (cc * bzu - rdx * (eR[c] - X[c]));
          if (!inside(c)) { Bx[c] = (R)0; Bz[c] = (R)0; }
        }
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const R en = c + 1 < C ? X[c + 1] : er;
          const R bxu = c + 1 < C ? Bx[c + 1] : bxr;
          const R bzu = c + 1 < C ? Bz[c + 1] : bzr;
          Bx[c] = a * Bx[c] + (cc * bxu + (en - X[c]));
          Bz[c] = a * Bz[c] + (cc * bzu - rdx * (eR[c] - X[c]));
          if (!inside(c)) { Bx[c] = (R)0; Bz[c] = (R)0; }
        }
      }
    }

    // ---- H'x^n = smx B_x + cb (D_k + D_k+1) (D at level n-1/2) into X; H'z^n = smz B_z into shared memory
    {
      R smx[C], smz[C], tmp[C];
      if (!mu_const) {
        lane_coefs<C, false, false>(I, A.tb, dq * (2 * n) - HALF_CELL + sxE, k0, liX, smx, tmp);
        lane_coefs<C, false, false>(I, A.tb, dq * (2 * n) + sxZ, k0, liZ, smz, tmp);
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) smx[c] = smz[c] = h0.x;
      }
      const R dr = __shfl_down_sync(FULL, D[0], 1);
#pragma unroll
      for (int c = 0; c < C; ++c) {
        const R d1 = c + 1 < C ? D[c + 1] : dr;
        X[c] = inside(c) ? smx[c] * Bx[c] + cb * (D[c] + d1) : (R)0;
        hz[c] = inside(c) ? smz[c] * Bz[c] : (R)0;
      }
      st_run<C, R>(sH + col * CELLS + lane * C, hz);
    }
    __syncthreads();

    // ---- D^{n+1/2}
    {
      const R hl = __shfl_up_sync(FULL, X[C - 1], 1);
      const R dl = __shfl_up_sync(FULL, D[C - 1], 1), dr = __shfl_down_sync(FULL, D[0], 1);
      R hL[C];
      ld_run<C, R>(sH + colL * CELLS + lane * C, hL);
      if (POS) {
#pragma unroll
        for (int c = C - 1; c >= 0; --c) {
          const R hp = c >= 1 ? X[c - 1] : hl;
          const R du = c >= 1 ? D[c - 1] : dl;
          D[c] = a * D[c] + (cc * du + ((X[c] - hp) - rdx * (hz[c] - hL[c])));
          if (!inside(c)) D[c] = (R)0;
        }
      } else {
#pragma unroll
        for (int c = 0; c < C; ++c) {
          const R hp = c >= 1 ? X[c - 1] : hl;
          const R du = c + 1 < C ? D[c + 1] : dr;
          D[c] = a * D[c] + (cc * du + ((X[c] - hp) - rdx * (hz[c] - hL[c])));
          if (!inside(c)) D[c] = (R)0;
        }
      }
    }

    // ---- line sources at t_{n+1/2}: D_{i,ks} += amp s(t) cos(kx x_i)
    for (unsigned m = smask; m; m &= m - 1) {
      const int q = __ffs(m) - 1;
      const int rel = A.srcs[q].node - base;
      if (lane == rel / C) {
        const R amp = (R)(A.src_amp[(long long)q * A.chunk_stride + A.s0 + s] * A.src_cos[q * A.nx + col]);
        const int cs = rel % C;
#pragma unroll
        for (int c = 0; c < C; ++c) D[c] += (c == cs) ? amp : (R)0;
      }
    }

    // ---- probes: E_y = D_y / eps at level n+1/2
    for (unsigned m = pmask; m; m &= m - 1) {
      const int q = __ffs(m) - 1;
      const int2 p = A.prb[q];
      const int rel = p.y - base;
      if (lane == rel / C) {
        R sep, cbp;
        node_coef<false, true>(I, A.tb, dq * (2 * n + 1) + sxE, p.y, sep, cbp);
        A.samples[(long long)q * A.chunk_stride + A.s0 + s] = (double)(pick(D, rel % C) * sep * (R)I.inv_S);
      }
    }
    // (the next step writes sE only after every warp has passed the barrier above,
    // and sH only after the next one, so the reads of this step are complete)
  }

  const int hi = min(x0 + W, (int)A.stride);
  store_cells<T, R, C>(A.Bx_out + row, k0, x0, hi, Bx);
  store_cells<T, R, C>(A.Bz_out + row, k0, x0, hi, Bz);
  store_cells<T, R, C>(A.D_out + row, k0, x0, hi, D);
}

// NXMAX: the largest column count the instantiation serves (its threads per
// block bound the registers a thread may use).
template <int C, int TB, bool POS, typename T, int NXMAX>
__global__ void __launch_bounds__(32 * NXMAX) te2d_kernel(const Args2D<T> A) {
  using R = typename Real<T>::type;
  constexpr int V = 16 / sizeof(T);
  constexpr int CELLS = 32 * C;
  extern __shared__ __align__(16) unsigned char smem2d[];
  R* sE = reinterpret_cast<R*>(smem2d);            // [column][cell] E'
  R* sH = sE + A.nx * CELLS;                         // [column][cell] H'z
  const InstDev I = *A.inst;
  const int x0 = A.tiles[blockIdx.x];
  const int base = x0 - tile_margin(TB, POS, V);
  if (base < 0 || base + CELLS > I.nz) te2d_tile<C, TB, POS, T, true>(A, I, x0, sE, sH);
  else te2d_tile<C, TB, POS, T, false>(A, I, x0, sE, sH);
}

template <int C, int TB, typename T, int NXMAX>
static int te2d_launch_cols(const Args2D<T>& a, bool pos, cudaStream_t st) {
  const size_t smem = 2 * sizeof(typename Real<T>::type) * (size_t)a.nx * 32 * C;
  const int threads = 32 * a.nx;
  if (pos) {
    cudaFuncSetAttribute(te2d_kernel<C, TB, true, T, NXMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    te2d_kernel<C, TB, true, T, NXMAX><<<a.n_tiles, threads, smem, st>>>(a);
  } else {
    cudaFuncSetAttribute(te2d_kernel<C, TB, false, T, NXMAX>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                         (int)smem);
    te2d_kernel<C, TB, false, T, NXMAX><<<a.n_tiles, threads, smem, st>>>(a);
  }
  return (int)cudaGetLastError();
}

template <int C, int TB, typename T>
static int te2d_launch_shape(const Args2D<T>& a, bool pos, cudaStream_t st) {
  if (a.nx <= 8) return te2d_launch_cols<C, TB, T, 8>(a, pos, st);
  if (a.nx <= 16) return te2d_launch_cols<C, TB, T, 16>(a, pos, st);
  return te2d_launch_cols<C, TB, T, 32>(a, pos, st);
}

// Tile shapes built (cells per lane, time block): FP32 8x8 and 8x16, FP64 8x8.
static bool shape_built(bool fp64, int C, int TB) {
  return C == 8 && (TB == 8 || (TB == 16 && !fp64));
}

template <typename T>
static int te2d_launch(int C, int TB, const Args2D<T>& a, bool pos, cudaStream_t st) {
  if (C == 8 && TB == 8) return te2d_launch_shape<8, 8, T>(a, pos, st);
  if constexpr (sizeof(T) == 4) {
    if (C == 8 && TB == 16) return te2d_launch_shape<8, 16, T>(a, pos, st);
  }
  return (int)cudaErrorInvalidValue;
}

}  // namespace gfdtd

using namespace gfdtd;

namespace {
constexpr int kChunk2D = 1024;

struct Buf2 {
  void* p = nullptr;
  size_t bytes = 0;
};

struct Probe2 {
  int i;
  long long k;
  std::vector<double> omega;
};
}  // namespace

struct gfdtd2d_ctx {
  int nx = 1;
  long long nz = 1, stride = 32;
  double dx = 1.0, S = 0.5;
  gfdtd_prec prec = GFDTD_F32;
  int eb = 4;
  cudaStream_t stream = nullptr;
  std::string err;
  // medium
  double beta = 0.0, slope = 0.0;
  std::vector<double> z, eps{1.0}, mu{1.0};
  std::vector<SrcDev> srcs;
  std::vector<double> kx;
  std::vector<Probe2> probes;
  // device
  Buf2 f[2][3];            // [parity][Bx, Bz, D]
  int cur = 0;
  long long n_done = 0;
  Buf2 d_ndone, d_inst, d_zq, d_tabE, d_tabH, d_tabE32, d_tabH32, d_srcs, d_amp, d_prb, d_prbdev,
      d_samples, d_omega, d_binprb, d_acc_re, d_acc_im, d_tiles, d_sx, d_srccos;
  int n_bins = 0;
  int C = 0, TB = 0;
  bool pos = true;
  int n_tiles = 0;
  bool dirty = true;
};

namespace {

gfdtd_status fail2(gfdtd2d_ctx* c, gfdtd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf;
  return s;
}

#define CK2(c, x)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess) return fail2(c, GFDTD_E_CUDA, "%s: %s", #x, cudaGetErrorString(e_)); \
  } while (0)

gfdtd_status alloc2(gfdtd2d_ctx* c, Buf2& b, size_t bytes) {
  if (b.p && b.bytes >= bytes) return GFDTD_OK;
  if (b.p) cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
  if (cudaMalloc(&b.p, std::max<size_t>(bytes, 16)) != cudaSuccess) {
    b.p = nullptr;
    cudaGetLastError();
    return fail2(c, GFDTD_E_OOM, "device allocation of %zu bytes failed", bytes);
  }
  b.bytes = std::max<size_t>(bytes, 16);
  return GFDTD_OK;
}

template <typename V>
gfdtd_status upload2(gfdtd2d_ctx* c, Buf2& b, const std::vector<V>& v) {
  gfdtd_status s = alloc2(c, b, v.size() * sizeof(V));
  if (s) return s;
  if (!v.empty()) CK2(c, cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice, c->stream));
  return GFDTD_OK;
}

gfdtd_status finalize2(gfdtd2d_ctx* c) {
  if (!c->dirty) return GFDTD_OK;
  // keep the DFT accumulators of probes that exist already
  std::vector<double> re(c->n_bins), im(c->n_bins);
  if (c->n_bins > 0) {
    CK2(c, cudaMemcpyAsync(re.data(), c->d_acc_re.p, re.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK2(c, cudaMemcpyAsync(im.data(), c->d_acc_im.p, im.size() * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK2(c, cudaStreamSynchronize(c->stream));
  }
  InstDev I{};
  I.nz = (int)c->nz;
  I.nz_pad = (int)c->stride;
  MediumSpec ms;
  ms.kind = 0;
  ms.beta = c->beta;
  ms.interp = 0;
  ms.n = (int)c->eps.size();
  ms.z = c->z.data();
  ms.eps = c->eps.data();
  ms.mu = c->mu.data();
  std::vector<long long> zq;
  std::vector<double2> tE, tH;
  std::vector<float2> tE32, tH32;
  fill_instance(ms, c->S, I, zq, tE, tH, tE32, tH32);
  c->pos = (I.flags & F_POS) != 0;
  std::vector<InstDev> iv{I};
  std::vector<int2> prb;
  std::vector<PrbDev> pd;
  std::vector<double> omega, acc_re, acc_im;
  std::vector<int> binprb;
  for (size_t p = 0; p < c->probes.size(); ++p) {
    const Probe2& q = c->probes[p];
    prb.push_back(make_int2(q.i, (int)q.k));
    PrbDev d;
    d.inst = 0;
    d.node = (int)q.k;
    d.nbins = (int)q.omega.size();
    d.bin0 = (int)omega.size();
    pd.push_back(d);
    for (double w : q.omega) {
      const size_t j = omega.size();
      omega.push_back(w);
      binprb.push_back((int)p);
      acc_re.push_back(j < re.size() ? re[j] : 0.0);
      acc_im.push_back(j < im.size() ? im[j] : 0.0);
    }
  }
  c->n_bins = (int)omega.size();
  gfdtd_status s;
  if ((s = upload2(c, c->d_inst, iv)) || (s = upload2(c, c->d_zq, zq)) || (s = upload2(c, c->d_tabE, tE)) ||
      (s = upload2(c, c->d_tabH, tH)) || (s = upload2(c, c->d_tabE32, tE32)) || (s = upload2(c, c->d_tabH32, tH32)) ||
      (s = upload2(c, c->d_srcs, c->srcs)) || (s = upload2(c, c->d_prb, prb)) ||
      (s = upload2(c, c->d_prbdev, pd)) || (s = upload2(c, c->d_omega, omega)) ||
      (s = upload2(c, c->d_binprb, binprb)) || (s = upload2(c, c->d_acc_re, acc_re)) ||
      (s = upload2(c, c->d_acc_im, acc_im)))
    return s;
  // per column: the slant offsets of its nodes and half nodes, and each source's cos(kx x_i)
  std::vector<long long> sx(2 * (size_t)c->nx);
  for (int i = 0; i < c->nx; ++i) {
    sx[2 * i] = llround(ldexp((double)i * c->dx * c->slope, 32));
    sx[2 * i + 1] = llround(ldexp(((double)i + 0.5) * c->dx * c->slope, 32));
  }
  std::vector<double> sc(std::max<size_t>(1, c->srcs.size() * c->nx));
  for (size_t q = 0; q < c->srcs.size(); ++q)
    for (int i = 0; i < c->nx; ++i) sc[q * c->nx + i] = std::cos(c->kx[q] * (double)i * c->dx);
  if ((s = upload2(c, c->d_sx, sx)) || (s = upload2(c, c->d_srccos, sc))) return s;
  if ((s = alloc2(c, c->d_amp, c->srcs.size() * kChunk2D * sizeof(double))) ||
      (s = alloc2(c, c->d_samples, c->probes.size() * kChunk2D * sizeof(double))))
    return s;
  if (c->C == 0) {
    c->C = 8;
    c->TB = c->prec == GFDTD_F64 ? 8 : 16;
  }
  const size_t smem = 2 * (size_t)c->eb * (size_t)c->nx * 32 * c->C;
  if (smem > 227 * 1024)
    return fail2(c, GFDTD_E_UNSUPPORTED, "tile %dx%d needs %zu bytes of shared memory for %d columns", c->C, c->TB,
                 smem, c->nx);
  const int V = 16 / c->eb;
  const int W = tile_width(c->C, c->TB, c->pos, V);
  std::vector<int> tiles;
  for (long long x0 = 0; x0 < c->nz; x0 += W) tiles.push_back((int)x0);
  c->n_tiles = (int)tiles.size();
  if ((s = upload2(c, c->d_tiles, tiles))) return s;
  c->dirty = false;
  return GFDTD_OK;
}

gfdtd_status check_field(gfdtd2d_ctx* c, int which) {
  if (which < 0 || which > 2) return fail2(c, GFDTD_E_ARG, "field must be 0 (D), 1 (B_x) or 2 (B_z)");
  return GFDTD_OK;
}

// buffer index of field `which` (0 D, 1 B_x, 2 B_z) in f[parity][Bx, Bz, D]
int slot(int which) { return which == 0 ? 2 : which - 1; }

template <typename T>
gfdtd_status step_chunk2d(gfdtd2d_ctx* c, int nsteps) {
  if (!c->srcs.empty()) {
    if (src_amp_launch((const SrcDev*)c->d_srcs.p, (int)c->srcs.size(), (double*)c->d_amp.p, kChunk2D, nsteps,
                       (const long long*)c->d_ndone.p, c->S, c->stream) != 0)
      return fail2(c, GFDTD_E_CUDA, "source amplitude launch failed");
  }
  for (int s0 = 0; s0 < nsteps; s0 += c->TB) {
    Args2D<T> a{};
    a.inst = (const InstDev*)c->d_inst.p;
    a.tb.zq = (const long long*)c->d_zq.p;
    a.tb.tabE = (const double2*)c->d_tabE.p;
    a.tb.tabH = (const double2*)c->d_tabH.p;
    a.tb.tabE32 = (const float2*)c->d_tabE32.p;
    a.tb.tabH32 = (const float2*)c->d_tabH32.p;
    a.nx = c->nx;
    a.stride = c->stride;
    a.inv_dx = 1.0 / c->dx;
    a.sx = (const long long*)c->d_sx.p;
    a.Bx_in = (const T*)c->f[c->cur][0].p;
    a.Bz_in = (const T*)c->f[c->cur][1].p;
    a.D_in = (const T*)c->f[c->cur][2].p;
    a.Bx_out = (T*)c->f[1 - c->cur][0].p;
    a.Bz_out = (T*)c->f[1 - c->cur][1].p;
    a.D_out = (T*)c->f[1 - c->cur][2].p;
    a.tiles = (const int*)c->d_tiles.p;
    a.n_tiles = c->n_tiles;
    a.srcs = (const SrcDev*)c->d_srcs.p;
    a.src_cos = (const double*)c->d_srccos.p;
    a.nsrc = (int)c->srcs.size();
    a.src_amp = (const double*)c->d_amp.p;
    a.prb = (const int2*)c->d_prb.p;
    a.nprb = (int)c->probes.size();
    a.samples = (double*)c->d_samples.p;
    a.chunk_stride = kChunk2D;
    a.n_done = (const long long*)c->d_ndone.p;
    a.s0 = s0;
    a.nsteps = std::min(c->TB, nsteps - s0);
    if (te2d_launch<T>(c->C, c->TB, a, c->pos, c->stream) != 0)
      return fail2(c, GFDTD_E_CUDA, "2D tile launch failed: %s", cudaGetErrorString(cudaGetLastError()));
    c->cur = 1 - c->cur;
  }
  if (c->n_bins > 0) {
    FoldArgs f;
    f.prbs = (const PrbDev*)c->d_prbdev.p;
    f.n_prb = (int)c->probes.size();
    f.samples = (const double*)c->d_samples.p;
    f.chunk_stride = kChunk2D;
    f.nsteps = nsteps;
    f.n_done = (const long long*)c->d_ndone.p;
    f.omega = (const double*)c->d_omega.p;
    f.bin_probe = (const int*)c->d_binprb.p;
    f.n_bins_total = c->n_bins;
    f.acc_re = (double*)c->d_acc_re.p;
    f.acc_im = (double*)c->d_acc_im.p;
    f.S = c->S;
    if (fold_launch(f, c->stream) != 0) return fail2(c, GFDTD_E_CUDA, "probe fold launch failed");
  }
  if (advance_launch((long long*)c->d_ndone.p, nsteps, c->stream) != 0)
    return fail2(c, GFDTD_E_CUDA, "step counter launch failed");
  c->n_done += nsteps;
  return GFDTD_OK;
}

}  // namespace

extern "C" {

gfdtd_status gfdtd2d_create(gfdtd2d_ctx** out, int nx, int64_t nz, double dx, double S, gfdtd_prec prec,
                            void* cuda_stream) {
  if (!out) return GFDTD_E_ARG;
  *out = nullptr;
  if (nx < 1 || nx > kMaxCols2D || nz < 1 || nz > (1LL << 26)) return GFDTD_E_ARG;
  if (!(dx > 0.0) || !std::isfinite(dx) || !(S > 0.0 && S <= 1.0)) return GFDTD_E_ARG;
  if (S * S * (1.0 + 1.0 / (dx * dx)) > 1.0) return GFDTD_E_ARG;   // 2D Yee limit in vacuum
  if (prec != GFDTD_F32 && prec != GFDTD_F64) return GFDTD_E_UNSUPPORTED;
  gfdtd2d_ctx* c = new (std::nothrow) gfdtd2d_ctx;
  if (!c) return GFDTD_E_OOM;
  c->nx = nx;
  c->nz = nz;
  c->stride = (nz + 31) / 32 * 32;
  c->dx = dx;
  c->S = S;
  c->prec = prec;
  c->eb = prec == GFDTD_F64 ? 8 : 4;
  c->stream = (cudaStream_t)cuda_stream;
  const size_t bytes = (size_t)c->eb * (size_t)nx * (size_t)c->stride;
  gfdtd_status s = GFDTD_OK;
  for (int p = 0; p < 2 && !s; ++p)
    for (int k = 0; k < 3 && !s; ++k) s = alloc2(c, c->f[p][k], bytes);
  if (!s) s = alloc2(c, c->d_ndone, 16);
  if (!s) {
    for (int p = 0; p < 2; ++p)
      for (int k = 0; k < 3; ++k) cudaMemsetAsync(c->f[p][k].p, 0, bytes, c->stream);
    cudaMemsetAsync(c->d_ndone.p, 0, 16, c->stream);
    if (cudaGetLastError() != cudaSuccess) s = GFDTD_E_CUDA;
  }
  if (s) {
    gfdtd2d_destroy(c);
    return s;
  }
  *out = c;
  return GFDTD_OK;
}

gfdtd_status gfdtd2d_set_medium(gfdtd2d_ctx* c, double beta, double slope, int n, const double* z,
                                const double* eps_r, const double* mu_r, int allow_unstable) {
  if (!c) return GFDTD_E_ARG;
  if (!(beta > -1.0 && beta < 1.0) || std::fabs(beta) * c->S >= 1.0) return fail2(c, GFDTD_E_ARG, "bad beta");
  if (!std::isfinite(slope)) return fail2(c, GFDTD_E_ARG, "bad slope");
  if (n < 1 || !eps_r || !mu_r || (n > 1 && !z)) return fail2(c, GFDTD_E_ARG, "need n >= 1 layers");
  for (int i = 0; i < n; ++i)
    if (!(eps_r[i] > 0.0) || !(mu_r[i] > 0.0)) return fail2(c, GFDTD_E_ARG, "eps and mu must be > 0");
  for (int i = 0; i + 1 < n; ++i) {
    if (!std::isfinite(z[i]) || std::fabs(z[i]) > 1e9) return fail2(c, GFDTD_E_ARG, "bad position");
    if (i > 0 && !(z[i] > z[i - 1])) return fail2(c, GFDTD_E_ARG, "positions must increase");
  }
  if (!allow_unstable)
    for (int i = 0; i < n; ++i)
      if (std::sqrt(eps_r[i] * mu_r[i]) * std::fabs(beta) > 1.0)
        return fail2(c, GFDTD_E_UNSTABLE, "layer %d: n|beta| > 1", i);
  c->beta = beta;
  c->slope = slope;
  c->z.assign(z ? z : eps_r, (z ? z : eps_r) + (z ? n - 1 : 0));
  c->eps.assign(eps_r, eps_r + n);
  c->mu.assign(mu_r, mu_r + n);
  c->dirty = true;
  return GFDTD_OK;
}

gfdtd_status gfdtd2d_add_source(gfdtd2d_ctx* c, int64_t k, double kx, double omega0, double tau, double t0,
                                double amp) {
  if (!c) return GFDTD_E_ARG;
  if (k < 0 || k >= c->nz || !(tau > 0.0) || !std::isfinite(kx) || !std::isfinite(omega0) || !std::isfinite(t0) ||
      !std::isfinite(amp))
    return fail2(c, GFDTD_E_ARG, "bad line source");
  if (c->srcs.size() >= 32) return fail2(c, GFDTD_E_ARG, "at most 32 line sources");
  SrcDev s{};
  s.inst = 0;
  s.node = (int)k;
  s.omega0 = omega0;
  s.tau = tau;
  s.t0 = t0;
  s.amp = amp;
  c->srcs.push_back(s);
  c->kx.push_back(kx);
  c->dirty = true;
  return GFDTD_OK;
}

gfdtd_status gfdtd2d_add_probe(gfdtd2d_ctx* c, int i, int64_t k, int n_bins, const double* omega, int* probe_id) {
  if (!c) return GFDTD_E_ARG;
  if (i < 0 || i >= c->nx || k < 0 || k >= c->nz || n_bins < 1 || !omega || !probe_id)
    return fail2(c, GFDTD_E_ARG, "bad probe");
  if (c->probes.size() >= 32) return fail2(c, GFDTD_E_ARG, "at most 32 probes");
  Probe2 p;
  p.i = i;
  p.k = k;
  p.omega.assign(omega, omega + n_bins);
  c->probes.push_back(p);
  *probe_id = (int)c->probes.size() - 1;
  c->dirty = true;
  return GFDTD_OK;
}

gfdtd_status gfdtd2d_set_tuning(gfdtd2d_ctx* c, int cells_per_lane, int time_block) {
  if (!c) return GFDTD_E_ARG;
  if (!shape_built(c->prec == GFDTD_F64, cells_per_lane, time_block))
    return fail2(c, GFDTD_E_UNSUPPORTED, "tile shape %dx%d not built", cells_per_lane, time_block);
  c->C = cells_per_lane;
  c->TB = time_block;
  c->dirty = true;
  return GFDTD_OK;
}

gfdtd_status gfdtd2d_step(gfdtd2d_ctx* c, int64_t n_steps) {
  if (!c || n_steps < 0) return GFDTD_E_ARG;
  gfdtd_status s = finalize2(c);
  if (s) return s;
  while (n_steps > 0) {
    const int ch = (int)std::min<int64_t>(n_steps, kChunk2D);
    s = c->prec == GFDTD_F64 ? step_chunk2d<double>(c, ch) : step_chunk2d<float>(c, ch);
    if (s) return s;
    n_steps -= ch;
  }
  return GFDTD_OK;
}

gfdtd_status gfdtd2d_read_fields(gfdtd2d_ctx* c, int which, double* host_dst, int64_t n) {
  if (!c || !host_dst) return GFDTD_E_ARG;
  gfdtd_status s = check_field(c, which);
  if (s) return s;
  if (n != (int64_t)c->nx * c->nz) return fail2(c, GFDTD_E_ARG, "n must be nx * nz");
  const size_t cnt = (size_t)c->nx * (size_t)c->stride;
  std::vector<double> tmp(cnt);
  std::vector<float> tf(c->prec == GFDTD_F64 ? 0 : cnt);
  void* dst = c->prec == GFDTD_F64 ? (void*)tmp.data() : (void*)tf.data();
  CK2(c, cudaMemcpyAsync(dst, c->f[c->cur][slot(which)].p, cnt * c->eb, cudaMemcpyDeviceToHost, c->stream));
  CK2(c, cudaStreamSynchronize(c->stream));
  for (int i = 0; i < c->nx; ++i)
    for (long long k = 0; k < c->nz; ++k) {
      const size_t src = (size_t)i * c->stride + k;
      host_dst[(size_t)i * c->nz + k] = c->prec == GFDTD_F64 ? tmp[src] : (double)tf[src];
    }
  return GFDTD_OK;
}

gfdtd_status gfdtd2d_write_fields(gfdtd2d_ctx* c, int which, const double* host_src, int64_t n) {
  if (!c || !host_src) return GFDTD_E_ARG;
  gfdtd_status s = check_field(c, which);
  if (s) return s;
  if (n != (int64_t)c->nx * c->nz) return fail2(c, GFDTD_E_ARG, "n must be nx * nz");
  const size_t cnt = (size_t)c->nx * (size_t)c->stride;
  std::vector<double> tmp(cnt, 0.0);
  std::vector<float> tf(cnt, 0.0f);
  for (int i = 0; i < c->nx; ++i)
    for (long long k = 0; k < c->nz; ++k) {
      const size_t d = (size_t)i * c->stride + k;
      tmp[d] = host_src[(size_t)i * c->nz + k];
      tf[d] = (float)tmp[d];
    }
  const void* src = c->prec == GFDTD_F64 ? (const void*)tmp.data() : (const void*)tf.data();
  CK2(c, cudaMemcpyAsync(c->f[c->cur][slot(which)].p, src, cnt * c->eb, cudaMemcpyHostToDevice, c->stream));
  CK2(c, cudaStreamSynchronize(c->stream));
  return GFDTD_OK;
}

gfdtd_status gfdtd2d_read_spectrum(gfdtd2d_ctx* c, int probe_id, double* re, double* im) {
  if (!c || !re || !im || probe_id < 0 || probe_id >= (int)c->probes.size()) return GFDTD_E_ARG;
  gfdtd_status s = finalize2(c);
  if (s) return s;
  int b0 = 0;
  for (int p = 0; p < probe_id; ++p) b0 += (int)c->probes[p].omega.size();
  const size_t nb = c->probes[probe_id].omega.size();
  CK2(c, cudaMemcpyAsync(re, (double*)c->d_acc_re.p + b0, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK2(c, cudaMemcpyAsync(im, (double*)c->d_acc_im.p + b0, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK2(c, cudaStreamSynchronize(c->stream));
  return GFDTD_OK;
}

gfdtd_status gfdtd2d_synchronize(gfdtd2d_ctx* c) {
  if (!c) return GFDTD_E_ARG;
  CK2(c, cudaStreamSynchronize(c->stream));
  return GFDTD_OK;
}

const char* gfdtd2d_last_error(const gfdtd2d_ctx* c) { return c ? c->err.c_str() : ""; }

void gfdtd2d_destroy(gfdtd2d_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  Buf2* bufs[] = {&c->d_ndone, &c->d_inst, &c->d_zq, &c->d_tabE, &c->d_tabH, &c->d_tabE32, &c->d_tabH32,
                  &c->d_srcs, &c->d_amp, &c->d_prb, &c->d_prbdev, &c->d_samples, &c->d_omega,
                  &c->d_binprb, &c->d_acc_re, &c->d_acc_im, &c->d_tiles, &c->d_sx, &c->d_srccos};
  for (Buf2* b : bufs)
    if (b->p) cudaFree(b->p);
  for (auto& p : c->f)
    for (auto& b : p)
      if (b.p) cudaFree(b.p);
  delete c;
}

}  // extern "C"
