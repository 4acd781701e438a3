// gfdtd_kernels.cu -- the plain one-step kernel, source amplitudes, running
// DFT probes, state conversions and the dispatch to the batched kernels.
#include "gfdtd_block.cuh"

namespace gfdtd {

int block_launch_f32(int, int, int, int, const void*, int, int, cudaStream_t);
int block_launch_f32w(int, int, int, int, const void*, int, int, cudaStream_t);
int block_launch_bf16(int, int, int, int, const void*, int, int, cudaStream_t);
int block_launch_f16(int, int, int, int, const void*, int, int, cudaStream_t);
int block_launch_f64(int, int, int, int, const void*, int, int, cudaStream_t);
int block_launch_f32k(int, int, int, int, const void*, int, int, cudaStream_t);
int block_occupancy_f32(int, int, int, int, int, int*);
int block_occupancy_f32w(int, int, int, int, int, int*);
int block_occupancy_bf16(int, int, int, int, int, int*);
int block_occupancy_f16(int, int, int, int, int, int*);
int block_occupancy_f64(int, int, int, int, int, int*);
int block_occupancy_f32k(int, int, int, int, int, int*);
int block_shapes_f32(int*, int*, int*, int);
int block_shapes_f32w(int*, int*, int*, int);
int block_shapes_bf16(int*, int*, int*, int);
int block_shapes_f16(int*, int*, int*, int);
int block_shapes_f64(int*, int*, int*, int);
int block_shapes_f32k(int*, int*, int*, int);

// prec takes the values of gfdtd_prec: 0 F32, 1 F32_KAHAN, 2 BF16, 3 F16, 4 F64.
int block_launch(int prec, int variant, int C, int TB, int MB, const void* args, int grid, int block,
                 cudaStream_t st) {
  switch (prec) {
    case 0: return C <= 16 ? block_launch_f32(variant, C, TB, MB, args, grid, block, st)
                           : block_launch_f32w(variant, C, TB, MB, args, grid, block, st);
    case 1: return block_launch_f32k(variant, C, TB, MB, args, grid, block, st);
    case 2: return block_launch_bf16(variant, C, TB, MB, args, grid, block, st);
    case 3: return block_launch_f16(variant, C, TB, MB, args, grid, block, st);
    case 4: return block_launch_f64(variant, C, TB, MB, args, grid, block, st);
  }
  return (int)cudaErrorInvalidValue;
}

int block_occupancy(int prec, int variant, int C, int TB, int MB, int block, int* nb) {
  switch (prec) {
    case 0: return C <= 16 ? block_occupancy_f32(variant, C, TB, MB, block, nb)
                           : block_occupancy_f32w(variant, C, TB, MB, block, nb);
    case 1: return block_occupancy_f32k(variant, C, TB, MB, block, nb);
    case 2: return block_occupancy_bf16(variant, C, TB, MB, block, nb);
    case 3: return block_occupancy_f16(variant, C, TB, MB, block, nb);
    case 4: return block_occupancy_f64(variant, C, TB, MB, block, nb);
  }
  return (int)cudaErrorInvalidValue;
}

int block_shapes(int prec, int* C, int* TB, int* MB, int max) {
  switch (prec) {
    case 0: {
      const int n = block_shapes_f32(C, TB, MB, max);
      return n + block_shapes_f32w(C + n, TB + n, MB + n, max - n);
    }
    case 1: return block_shapes_f32k(C, TB, MB, max);
    case 2: return block_shapes_bf16(C, TB, MB, max);
    case 3: return block_shapes_f16(C, TB, MB, max);
    case 4: return block_shapes_f64(C, TB, MB, max);
  }
  return 0;
}

// ------------------------------------------------------------ plain kernel
//
// One step of one instance per launch, fields in HBM: the throughput baseline
// of the batched kernel.  Thread t of a block of 256 holds cell k0 - 4 + t:
// it stages that cell's old B and D in shared memory, forms E' there (cells
// k0 - 2 .. k0 + 250), then B' and, from its own B', H' (k0 - 2 .. k0 + 249
// and k0 - 1 .. k0 + 248), then D' (k0 .. k0 + 248, the block's 249 output
// cells; B' at k0 + 249 serves a probe's average at k0 + 248), a barrier
// between the three stages, so that each intermediate value is formed once.  The instance record travels in the launch parameters.
// The material: in one coalesced pass that waits on no other load, the block
// reads the instance's profile (positions and both coefficient tables), keeps
// its first kPlainP entries in shared memory and counts, for each of the two
// levels, the positions left of its first staged cell and those left of its
// last one; a cell then finds its entry by a binary search between those two
// counts.  So the field loads and that pass are the only global reads before
// the stores (entries past kPlainP, in longer profiles, are read from global
// memory where a search reaches them).
constexpr int kPlainP = 512;
constexpr int kPlainThreads = 256, kPlainOut = kPlainThreads - 7;

template <typename R>
struct PlainProfile {
  using V = typename TabOf<R>::V;
  long long z[kPlainP];
  V vE[kPlainP], vH[kPlainP];
  int loE, hiE, loH, hiH;        // counts at the first and at the last staged cell
};

template <typename R>
struct PlainTab {
  using V = typename TabOf<R>::V;
  const PlainProfile<R>& P;
  const long long* __restrict__ zq;
  const V* __restrict__ tE;
  const V* __restrict__ tH;
  __device__ __forceinline__ long long z(int i) const { return i < kPlainP ? P.z[i] : __ldg(zq + i); }
  __device__ __forceinline__ V v(bool eside, int i) const {
    if (i < kPlainP) return eside ? P.vE[i] : P.vH[i];
    return __ldg((eside ? tE : tH) + i);
  }
  // number of positions at or left of node k, given that it lies in [lo, hi]
  __device__ __forceinline__ int count(long long off, int k, int lo, int hi) const {
    while (lo < hi) {
      const int m = (lo + hi) >> 1;
      if (node_of(z(m), off) <= k) lo = m + 1; else hi = m;
    }
    return lo;
  }
};

template <typename R>
struct PlainShared {
  R B[kPlainThreads], D[kPlainThreads], E[kPlainThreads], Bn[kPlainThreads], H[kPlainThreads];
  PlainProfile<R> P;
};

template <bool MATTER, bool ESIDE, typename R>
__device__ __forceinline__ void plain_coef(const InstDev& I, const PlainTab<R>& T, long long off, int k,
                                           int idx, R& cx, R& cy) {
  if (!(I.flags & F_LINEAR)) {
    const auto v = T.v(ESIDE, idx);
    cx = v.x;
    cy = MATTER ? v.y : coef<R>(I.cb, I.cb32);
    return;
  }
  const int n = I.n;
  R e, m;
  if (idx <= 0 || idx >= n) {
    const auto v = T.v(true, idx <= 0 ? 0 : n - 1);
    e = v.x;
    m = v.y;
  } else {
    const long long z0 = T.z(idx - 1), z1 = T.z(idx);
    const long long xi = ((long long)k << 32) - off;
    const R wgt = (R)(xi - z0) / (R)(z1 - z0);
    const auto v0 = T.v(true, idx - 1), v1 = T.v(true, idx);
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

template <bool MATTER, typename T>
__device__ void plain_block(const PlainArgs<T>& A, PlainShared<typename Real<T>::type>& sh) {
  using R = typename Real<T>::type;
  constexpr int NT = kPlainThreads, H = 4;
  PlainProfile<R>& P = sh.P;
  const InstDev& I = A.I;
  const int nz = I.nz;
  const int k0 = blockIdx.x * kPlainOut;
  const int t = threadIdx.x;
  const int k = k0 - H + t;                // this thread's cell
  const bool in = k >= 0 && k < nz;
  const bool pos = (I.flags & F_POS) != 0;
  const R a = coef<R>(I.a, I.a32), cc = coef<R>(I.c, I.c32);
  const int sc = *A.s_dev;                 // step within the chunk
  const long long n = *A.n_done + sc + 1;
  const long long offE = I.dq * (2 * n - 1), offH = I.dq * (2 * n) - HALF_CELL;
  const PlainTab<R> tab{P, A.tb.zq + I.tab, TabOf<R>::get(A.tb, true) + I.tab, TabOf<R>::get(A.tb, false) + I.tab};

  sh.B[t] = in ? (R)A.Bin[I.off + k] : (R)0;
  sh.D[t] = in ? (R)A.Din[I.off + k] : (R)0;
  const int nbp = (I.flags & F_LINEAR) ? I.n : I.n - 1;   // positions (the tables hold I.n entries)
  {
    const int klo = k0 - H, khi = k0 - H + NT - 1;
    int loE = 0, hiE = 0, loH = 0, hiH = 0;
    for (int j0 = 0; j0 < I.n; j0 += NT) {
      const int jj = j0 + t;
      bool pl = false, ph = false, ql = false, qh = false;
      if (jj < I.n && jj < kPlainP) {
        P.vE[jj] = __ldg(tab.tE + jj);
        P.vH[jj] = __ldg(tab.tH + jj);
      }
      if (jj < nbp) {
        const long long z = __ldg(tab.zq + jj);
        if (jj < kPlainP) P.z[jj] = z;
        const int kE = node_of(z, offE), kH = node_of(z, offH);
        pl = kE <= klo;
        ph = kE <= khi;
        ql = kH <= klo;
        qh = kH <= khi;
      }
      loE += __syncthreads_count(pl);
      hiE += __syncthreads_count(ph);
      loH += __syncthreads_count(ql);
      hiH += __syncthreads_count(qh);
    }
    if (t == 0) {
      P.loE = loE;
      P.hiE = hiE;
      P.loH = loH;
      P.hiH = hiH;
    }
  }
  __syncthreads();

  // E'^{n-1/2} at cells k0 - 2 .. k0 + 250 (B at level n-1)
  if (t >= 2 && t <= NT - 2) {
    R e = (R)0;
    if (in) {
      R se, cb;
      plain_coef<MATTER, true>(I, tab, offE, k, tab.count(offE, k, P.loE, P.hiE), se, cb);
      const R bs = pos ? sh.B[t - 1] + sh.B[t - 2] : sh.B[t] + sh.B[t + 1];
      e = se * sh.D[t] - cb * bs;
    }
    sh.E[t] = e;
  }
  __syncthreads();

  // B^n at cells k0 - 2 .. k0 + 249 (absorbing layers damp after the update), and
  // from it H'^n at k0 - 1 .. k0 + 248 (D at level n-1/2)
  if (t >= 2 && t <= NT - 3) {
    R b = (R)0, h = (R)0;
    if (in) {
      const R bu = pos ? sh.B[t - 1] : sh.B[t + 1];
      b = a * sh.B[t] + (cc * bu + (sh.E[t] - sh.E[t + 1]));
      if (I.abs_w > 0) b *= absorb_factor<R>(I, (R)k + (R)0.5);
      if (t >= 3 && t <= NT - 4) {
        R sm, cb;
        plain_coef<MATTER, false>(I, tab, offH, k, tab.count(offH, k, P.loH, P.hiH), sm, cb);
        h = sm * b - cb * (sh.D[t] + sh.D[t + 1]);
      }
      if (t >= H && t <= NT - 4) A.Bout[I.off + k] = (T)b;
    }
    sh.Bn[t] = b;
    sh.H[t] = h;
  }
  __syncthreads();

  // D^{n+1/2} at the block's output cells k0 .. k0 + 248, sources and probes
  if (t < H || t > NT - 4 || !in) return;
  const R du = pos ? sh.D[t - 1] : sh.D[t + 1];
  R d = a * sh.D[t] + (cc * du + (sh.H[t - 1] - sh.H[t]));
  if (I.abs_w > 0) d *= absorb_factor<R>(I, (R)k);
  for (int q = 0; q < I.nsrc; ++q)   // amplitudes at t_{n+1/2}, formed once per chunk
    if (A.srcs[I.src0 + q].node == k) d += (R)A.src_amp[(long long)(I.src0 + q) * A.chunk_stride + sc];
  for (int q = 0; q < I.nprb; ++q) {
    if (A.prbs[I.prb0 + q].node == k) {
      const long long offP = I.dq * (2 * n + 1);
      R se, cb;
      plain_coef<MATTER, true>(I, tab, offP, k, tab.count(offP, k, 0, nbp), se, cb);
      R F = d * se;
      if (MATTER) {
        const R bbar = pos ? (R)0.5 * (sh.Bn[t - 1] + sh.Bn[t - 2]) : (R)0.5 * (sh.Bn[t] + sh.Bn[t + 1]);
        F += ((R)I.beta * (R)I.S - (R)2 * cb) * bbar;
      }
      A.samples[(long long)(I.prb0 + q) * A.chunk_stride + sc] = (double)(F * (R)I.inv_S);
    }
  }
  A.Dout[I.off + k] = (T)d;
}

template <typename T>
__global__ void __launch_bounds__(kPlainThreads) plain_kernel(const PlainArgs<T> A) {
  __shared__ PlainShared<typename Real<T>::type> sh;
  if (A.I.flags & F_MATTER) plain_block<true>(A, sh);
  else plain_block<false>(A, sh);
}

// The launch structure of the plain path without its arithmetic (gfdtd_plain_floor):
// the plain kernel's grid, every thread reads its cell's B and D, the block's
// output cells are written back unchanged (U: an unsigned type of the element's size).
template <typename U>
__global__ void __launch_bounds__(kPlainThreads) plain_floor_kernel(U* B, U* D, int nz, const int* s_dev) {
  const int t = threadIdx.x;
  const int k = blockIdx.x * kPlainOut - 4 + t;
  if (*s_dev < 0 || k < 0 || k >= nz) return;
  volatile U* vB = B;
  volatile U* vD = D;
  const U b = vB[k], d = vD[k];
  if (t >= 4 && t <= kPlainThreads - 4) {
    vB[k] = b;
    vD[k] = d;
  }
}

int plain_floor_launch(int elem_bytes, void* B, void* D, int nz, const int* s_dev, cudaStream_t st) {
  const int grid = (nz + kPlainOut - 1) / kPlainOut;
  switch (elem_bytes) {
    case 2: plain_floor_kernel<unsigned short><<<grid, kPlainThreads, 0, st>>>((unsigned short*)B, (unsigned short*)D, nz, s_dev); break;
    case 4: plain_floor_kernel<unsigned><<<grid, kPlainThreads, 0, st>>>((unsigned*)B, (unsigned*)D, nz, s_dev); break;
    case 8: plain_floor_kernel<unsigned long long><<<grid, kPlainThreads, 0, st>>>((unsigned long long*)B, (unsigned long long*)D, nz, s_dev); break;
    default: return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

__global__ void plain_tick_kernel(int* s_dev) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *s_dev += 1;
}

int plain_tick_launch(int* s_dev, cudaStream_t st) {
  plain_tick_kernel<<<1, 32, 0, st>>>(s_dev);
  return (int)cudaGetLastError();
}

template <typename T>
static int plain_t(const void* args, int nz, cudaStream_t st) {
  plain_kernel<T><<<(nz + kPlainOut - 1) / kPlainOut, kPlainThreads, 0, st>>>(*static_cast<const PlainArgs<T>*>(args));
  return (int)cudaGetLastError();
}

int plain_launch(int prec, const void* args, int nz, cudaStream_t st) {
  switch (prec) {
    case 0: return plain_t<float>(args, nz, st);
    case 2: return plain_t<__nv_bfloat16>(args, nz, st);
    case 3: return plain_t<__half>(args, nz, st);
    case 4: return plain_t<double>(args, nz, st);
  }
  return (int)cudaErrorInvalidValue;
}

// ------------------------------------------------- sources, DFT, bookkeeping

// Source amplitudes of one chunk of steps, s(t_{n+1/2}) for n = n_done + 1 ...
__global__ void src_amp_kernel(const SrcDev* srcs, int nsrc, double* amp, int stride, int nsteps,
                               const long long* n_done, double S) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nsrc * nsteps) return;
  const int q = i / nsteps, s = i % nsteps;
  const long long n = *n_done + s + 1;
  const SrcDev sd = srcs[q];
  const double t = (double)(2 * n + 1) * S * 0.5;
  const double u = t - sd.t0;
  amp[(long long)q * stride + s] = sd.amp * sin(sd.omega0 * u) * exp(-(u / sd.tau) * (u / sd.tau));
}

int src_amp_launch(const SrcDev* srcs, int nsrc, double* amp, int stride, int nsteps,
                   const long long* n_done, double S, cudaStream_t st) {
  const int total = nsrc * nsteps;
  if (total == 0) return 0;
  src_amp_kernel<<<(total + 255) / 256, 256, 0, st>>>(srcs, nsrc, amp, stride, nsteps, n_done, S);
  return (int)cudaGetLastError();
}

// X(w) += sum_s F_s exp(i w t_s) S over one chunk of samples, one thread per
// bin.  The phasor advances by a fixed rotation exp(i w S) and is recomputed
// directly every 64 samples, so its error stays at the level of FP64 rounding.
__global__ void fold_kernel(const FoldArgs A) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= A.n_bins_total) return;
  const int p = A.bin_probe[b];
  const double* __restrict__ f = A.samples + (long long)p * A.chunk_stride;
  const double w = A.omega[b];
  const long long n1 = *A.n_done + 1;
  double rs, rc;
  sincos(w * A.S, &rs, &rc);
  double re = 0.0, im = 0.0, pc = 0.0, ps = 0.0;
  for (int s = 0; s < A.nsteps; ++s) {
    if ((s & 63) == 0) {
      const double t = (double)(2 * (n1 + s) + 1) * A.S * 0.5;
      sincos(w * t, &ps, &pc);
    } else {
      const double nc = pc * rc - ps * rs;
      ps = ps * rc + pc * rs;
      pc = nc;
    }
    const double F = __ldg(f + s);
    re = fma(F, pc, re);
    im = fma(F, ps, im);
  }
  A.acc_re[b] += re * A.S;
  A.acc_im[b] += im * A.S;
}

int fold_launch(const FoldArgs& a, cudaStream_t st) {
  if (a.n_bins_total == 0 || a.nsteps == 0) return 0;
  fold_kernel<<<(a.n_bins_total + 127) / 128, 128, 0, st>>>(a);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------ watchdog
//
// The scheme is unstable where n|beta| > 1 (Sec. 5); an instance run there
// grows until it overflows.  Once per chunk this scan reads the state (B, D) and
// merges, per instance, the largest magnitude into one word: the bits of
// |x| rounded to FP32, which order like the values and put infinities
// (0x7f800000) and NaNs above every finite value, so one integer maximum also
// records a non-finite value.  A separate pass, not a step inside the tile
// kernels: it reads 2 values per cell once per chunk (under 1 % of the
// batched kernel's traffic), where the same reduction inside the fast kernel's
// tiles cost it 13 % on the crystal.
constexpr int kWatchThreads = 256;

template <typename T>
__global__ void __launch_bounds__(kWatchThreads) watch_kernel(const WatchBlock* __restrict__ blocks,
                                                              const T* __restrict__ B, const T* __restrict__ D,
                                                              unsigned* __restrict__ watch) {
  using R = typename Real<T>::type;
  constexpr int V = 16 / sizeof(T);
  const WatchBlock wb = blocks[blockIdx.x];
  unsigned m = 0u;
  for (long long e = wb.start + (long long)threadIdx.x * V; e < wb.end; e += (long long)kWatchThreads * V) {
    R x[V];
    unpack(__ldg(reinterpret_cast<const uint4*>(B + e)), x, T());
#pragma unroll
    for (int j = 0; j < V; ++j) m = max(m, __float_as_uint((float)x[j]) & 0x7fffffffu);
    unpack(__ldg(reinterpret_cast<const uint4*>(D + e)), x, T());
#pragma unroll
    for (int j = 0; j < V; ++j) m = max(m, __float_as_uint((float)x[j]) & 0x7fffffffu);
  }
  m = __reduce_max_sync(FULL, m);
  __shared__ unsigned sm[kWatchThreads / 32];
  if ((threadIdx.x & 31) == 0) sm[threadIdx.x >> 5] = m;
  __syncthreads();
  if (threadIdx.x == 0) {
    for (int w = 1; w < kWatchThreads / 32; ++w) m = max(m, sm[w]);
    if (m != 0u) atomicMax(watch + wb.inst, m);
  }
}

int watch_launch(int prec, const WatchBlock* blocks, int n_blocks, const void* B, const void* D,
                 unsigned* watch, cudaStream_t st) {
  if (n_blocks == 0) return 0;
  switch (prec) {
    case 0: case 1:
      watch_kernel<float><<<n_blocks, kWatchThreads, 0, st>>>(blocks, (const float*)B, (const float*)D, watch);
      break;
    case 2:
      watch_kernel<__nv_bfloat16><<<n_blocks, kWatchThreads, 0, st>>>(blocks, (const __nv_bfloat16*)B,
                                                                       (const __nv_bfloat16*)D, watch);
      break;
    case 3:
      watch_kernel<__half><<<n_blocks, kWatchThreads, 0, st>>>(blocks, (const __half*)B, (const __half*)D, watch);
      break;
    case 4:
      watch_kernel<double><<<n_blocks, kWatchThreads, 0, st>>>(blocks, (const double*)B, (const double*)D, watch);
      break;
    default:
      return (int)cudaErrorInvalidValue;
  }
  return (int)cudaGetLastError();
}

__global__ void advance_kernel(long long* n_done, long long by) {
  if (threadIdx.x == 0 && blockIdx.x == 0) *n_done += by;
}

int advance_launch(long long* n_done, long long by, cudaStream_t st) {
  advance_kernel<<<1, 32, 0, st>>>(n_done, by);
  return (int)cudaGetLastError();
}

// ------------------------------------------------------------- conversions

template <typename T>
__global__ void to_double_kernel(const T* src, double* dst, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (double)(typename Real<T>::type)src[i];
}
template <typename T>
__global__ void from_double_kernel(const double* src, T* dst, long long n) {
  const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
  if (i < n) dst[i] = (T)(typename Real<T>::type)src[i];
}

template <typename T>
static int convert_t(int to_double, const void* src, void* dst, long long n, cudaStream_t st) {
  if (n == 0) return 0;
  const unsigned blocks = (unsigned)((n + 255) / 256);
  if (to_double) to_double_kernel<T><<<blocks, 256, 0, st>>>((const T*)src, (double*)dst, n);
  else from_double_kernel<T><<<blocks, 256, 0, st>>>((const double*)src, (T*)dst, n);
  return (int)cudaGetLastError();
}

int convert_launch(int prec, int to_double, const void* src, void* dst, long long n, cudaStream_t st) {
  switch (prec) {
    case 0: case 1: return convert_t<float>(to_double, src, dst, n, st);
    case 2: return convert_t<__nv_bfloat16>(to_double, src, dst, n, st);
    case 3: return convert_t<__half>(to_double, src, dst, n, st);
    case 4: return convert_t<double>(to_double, src, dst, n, st);
  }
  return (int)cudaErrorInvalidValue;
}

// Derived fields of one instance at the state (B^n, D^{n+1/2}), in FP64:
// which 2 = E (level n+1/2), 3 = H (level n, moving perturbation), 4 = E*.
template <bool MATTER, typename T>
__device__ double derived_value(int which, const InstDev& I, const Tables& tb, const T* Bi, const T* Di,
                                long long n, int k) {
  using R = typename Real<T>::type;
  auto ld = [&](const T* p, int j) -> double {
    return (j >= 0 && j < I.nz) ? (double)(R)p[j] : 0.0;
  };
  if (which == 3) {
    double sm, cb;
    node_coef<MATTER, false>(I, tb, I.dq * (2 * n) - HALF_CELL, k, sm, cb);
    return ld(Bi, k) * sm / I.S;
  }
  double se, cb;
  node_coef<MATTER, true>(I, tb, I.dq * (2 * n + 1), k, se, cb);
  const bool pos = (I.flags & F_POS) != 0;
  const double bbar = pos ? 0.5 * (ld(Bi, k - 1) + ld(Bi, k - 2)) : 0.5 * (ld(Bi, k) + ld(Bi, k + 1));
  const double estar = (se * ld(Di, k) - 2.0 * cb * bbar) / I.S;
  return which == 4 ? estar : estar + I.beta * bbar;
}

template <bool MATTER, typename T>
__device__ void derived_cell(int which, const InstDev& I, const Tables& tb, const T* Bi,
                             const T* Di, double* out, long long n, int k) {
  out[k] = derived_value<MATTER, T>(which, I, tb, Bi, Di, n, k);
}

template <typename T>
__global__ void derived_kernel(int which, const InstDev* inst, int i, Tables tb, const T* B,
                               const T* D, double* out, long long n) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const InstDev I = inst[i];
  if (k >= I.nz) return;
  if (I.flags & F_MATTER) derived_cell<true>(which, I, tb, B + I.off, D + I.off, out, n, k);
  else derived_cell<false>(which, I, tb, B + I.off, D + I.off, out, n, k);
}

template <typename T>
static int derived_t(int which, const InstDev* inst, int i, Tables tb, const void* B, const void* D,
                     double* out, int nz, long long n, cudaStream_t st) {
  derived_kernel<T><<<(nz + 255) / 256, 256, 0, st>>>(which, inst, i, tb, (const T*)B, (const T*)D,
                                                      out, n);
  return (int)cudaGetLastError();
}

int derived_launch(int prec, int which, const InstDev* inst, int i, Tables tb, const void* B,
                   const void* D, double* out, int nz, long long n, cudaStream_t st) {
  switch (prec) {
    case 0: case 1: return derived_t<float>(which, inst, i, tb, B, D, out, nz, n, st);
    case 2: return derived_t<__nv_bfloat16>(which, inst, i, tb, B, D, out, nz, n, st);
    case 3: return derived_t<__half>(which, inst, i, tb, B, D, out, nz, n, st);
    case 4: return derived_t<double>(which, inst, i, tb, B, D, out, nz, n, st);
  }
  return (int)cudaErrorInvalidValue;
}

// ------------------------------------------------------------ space-time capture
//
// One frame: field `which` (0 D, 1 B, 2 E, 3 H, 4 E*) of instance i at the
// state (B^n, D^{n+1/2}), at cells z0 + j zs, j < m, stored as FP32 or FP16.

__device__ __forceinline__ void store_frame(float* o, long long j, double v) { o[j] = (float)v; }
__device__ __forceinline__ void store_frame(__half* o, long long j, double v) { o[j] = __double2half(v); }

template <typename T, typename O>
__global__ void capture_kernel(int which, const InstDev* inst, int i, Tables tb, const T* B, const T* D,
                               long long z0, long long zs, long long m, long long n, O* out) {
  using R = typename Real<T>::type;
  const long long j = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (j >= m) return;
  const InstDev I = inst[i];
  const int k = (int)(z0 + j * zs);
  double v;
  if (which == 0) v = (double)(R)D[I.off + k];
  else if (which == 1) v = (double)(R)B[I.off + k];
  else if (I.flags & F_MATTER) v = derived_value<true, T>(which, I, tb, B + I.off, D + I.off, n, k);
  else v = derived_value<false, T>(which, I, tb, B + I.off, D + I.off, n, k);
  store_frame(out, j, v);
}

template <typename T>
static int capture_t(int which, const InstDev* inst, int i, Tables tb, const void* B, const void* D,
                     long long z0, long long zs, long long m, long long n, int half, void* out,
                     cudaStream_t st) {
  const unsigned grid = (unsigned)((m + 255) / 256);
  if (half)
    capture_kernel<T, __half><<<grid, 256, 0, st>>>(which, inst, i, tb, (const T*)B, (const T*)D, z0, zs, m, n,
                                                    (__half*)out);
  else
    capture_kernel<T, float><<<grid, 256, 0, st>>>(which, inst, i, tb, (const T*)B, (const T*)D, z0, zs, m, n,
                                                   (float*)out);
  return (int)cudaGetLastError();
}

int capture_launch(int prec, int which, const InstDev* inst, int i, Tables tb, const void* B, const void* D,
                   long long z0, long long zs, long long m, long long n, int half, void* out, cudaStream_t st) {
  switch (prec) {
    case 0: case 1: return capture_t<float>(which, inst, i, tb, B, D, z0, zs, m, n, half, out, st);
    case 2: return capture_t<__nv_bfloat16>(which, inst, i, tb, B, D, z0, zs, m, n, half, out, st);
    case 3: return capture_t<__half>(which, inst, i, tb, B, D, z0, zs, m, n, half, out, st);
    case 4: return capture_t<double>(which, inst, i, tb, B, D, z0, zs, m, n, half, out, st);
  }
  return (int)cudaErrorInvalidValue;
}

// ---------------------------------------------------------------- one-way sources

// One block per one-way source advances its auxiliary grid (the same leapfrog
// step as the batched kernels, in the arithmetic type R: FP64 for FP64 fields,
// FP32 otherwise -- GB300's FP64 rate made an FP64 grid per source cost more
// than the batch it drives; uniform background, graded layers at
// both ends, soft source at kTfsfAuxSrc) through the chunk's steps in shared
// memory, and writes for every step the additive corrections that make the
// main grid's cells node-2 .. node+1 read each neighbour in their own region's
// convention (total field at nodes >= node, scattered field left of it):
//   v >= 0: B_{q-1} += S ie Di_q,  B_q += -S hb Bi_{q-2} + beta S Bi_{q-1},  B_{q+1} += -S hb Bi_{q-1};
//   v <  0: B_{q-2} += -S hb Bi_q, B_{q-1} += S ie Di_q - S hb Bi_{q+1} + beta S Bi_q;
//   D_{q-1} += -S hb Di_q (+ beta S Di_q for v < 0),
//   D_q += S (im Bn_{q-1} - hb Di_{q-1}) (+ beta S Di_{q-1} for v >= 0),
// with Bi, Di the incident B^{n-1}, D^{n-1/2} and Bn the incident B^n (aux
// cell = main cell - q + kTfsfAuxQ).
constexpr int kTfsfThreads = 256;   // one block per source: several blocks share an SM

template <typename R>
__global__ void __launch_bounds__(kTfsfThreads, 4) tfsf_aux_kernel(const TfsfDev* __restrict__ tfs, R* __restrict__ aux,
                                                                double* __restrict__ corr, int chunk_stride,
                                                                const long long* __restrict__ n_done, int nsteps) {
  constexpr int N = kTfsfAuxN, Q = kTfsfAuxQ;
  constexpr int PER = (N + kTfsfThreads - 1) / kTfsfThreads;   // cells per thread
  __shared__ R sB[N], sD[N], sE[N], sH[N];
  const TfsfDev tf = tfs[blockIdx.x];
  R* gB = aux + (size_t)blockIdx.x * 2 * kTfsfAuxPad;
  R* gD = gB + kTfsfAuxPad;
  const int tid = threadIdx.x, nt = kTfsfThreads;
  for (int i = tid; i < N; i += nt) { sB[i] = gB[i]; sD[i] = gD[i]; }
  const R S = (R)tf.S, beta = (R)tf.beta, ie = (R)tf.ie, im = (R)tf.im, hb = (R)tf.hb;
  const bool pos = beta >= 0.0;
  // damping factors of this thread's cells: exp(-sigma d^2), d the depth into a layer / its width
  R fB[PER], fD[PER];
#pragma unroll
  for (int j = 0; j < PER; ++j) {
    const int i = tid + j * nt;
    auto f = [&](double x) {
      const double W = (double)kTfsfAuxW, right = (double)(N - 1) - W;
      double d = 0.0;
      if (x < W) d = (W - x) / W;
      else if (x > right) d = (x - right) / W;
      return (R)exp(-kTfsfAuxSigma * d * d);
    };
    fB[j] = f((double)i + 0.5);
    fD[j] = f((double)i);
  }
  auto at = [&](const R* a, int i) { return (i < 0 || i >= N) ? (R)0 : a[i]; };
  const long long n0 = *n_done;
  double* out = corr + (size_t)blockIdx.x * chunk_stride * kTfsfCorr;
  __syncthreads();
  for (int s = 0; s < nsteps; ++s) {
    const long long n = n0 + s + 1;
    R Bm2 = 0, Bm1 = 0, B0 = 0, Bp1 = 0, Dm1 = 0, D0 = 0;
    if (tid == 0) { Bm2 = sB[Q - 2]; Bm1 = sB[Q - 1]; B0 = sB[Q]; Bp1 = sB[Q + 1]; Dm1 = sD[Q - 1]; D0 = sD[Q]; }
    // E*^{n-1/2} = ie D - 2 hb Bbar (B at level n-1)
    for (int i = tid; i < N; i += nt) {
      const R bbar = pos ? (R)0.5 * (at(sB, i - 1) + at(sB, i - 2)) : (R)0.5 * (at(sB, i + 1) + sB[i]);
      sE[i] = ie * sD[i] - (R)2 * hb * bbar;
    }
    __syncthreads();
    R nb[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = tid + j * nt;
      if (i < N) {
        const R dB = pos ? sB[i] - at(sB, i - 1) : at(sB, i + 1) - sB[i];
        nb[j] = (sB[i] - S * (at(sE, i + 1) - sE[i]) - beta * S * dB) * fB[j];
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) { const int i = tid + j * nt; if (i < N) sB[i] = nb[j]; }
    __syncthreads();
    // H*^n = im B^n - hb (D_j + D_{j+1}) (D at level n-1/2)
    for (int i = tid; i < N; i += nt) sH[i] = im * sB[i] - hb * (sD[i] + at(sD, i + 1));
    __syncthreads();
    R nd[PER];
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = tid + j * nt;
      if (i < N) {
        const R dD = pos ? sD[i] - at(sD, i - 1) : at(sD, i + 1) - sD[i];
        nd[j] = (sD[i] - S * (sH[i] - at(sH, i - 1)) - beta * S * dD) * fD[j];
      }
    }
    __syncthreads();
#pragma unroll
    for (int j = 0; j < PER; ++j) {
      const int i = tid + j * nt;
      if (i < N) {
        R d = nd[j];
        if (i == kTfsfAuxSrc) {   // the source waveform in FP64, as for soft sources
          const double u = (double)(2 * n + 1) * tf.S * 0.5 - tf.t0;
          d += (R)(tf.amp * sin(tf.omega0 * u) * exp(-(u / tf.tau) * (u / tf.tau)));
        }
        sD[i] = d;
      }
    }
    __syncthreads();
    if (tid == 0) {
      const R Bn = sB[Q - 1];
      double* c = out + (size_t)s * kTfsfCorr;
      if (pos) {
        c[0] = 0.0;
        c[1] = S * ie * D0;
        c[2] = -S * hb * Bm2 + beta * S * Bm1;
        c[3] = -S * hb * Bm1;
        c[4] = -S * hb * D0;
        c[5] = S * (im * Bn - hb * Dm1) + beta * S * Dm1;
      } else {
        c[0] = -S * hb * B0;
        c[1] = S * ie * D0 - S * hb * Bp1 + beta * S * B0;
        c[2] = 0.0;
        c[3] = 0.0;
        c[4] = -S * hb * D0 + beta * S * D0;
        c[5] = S * (im * Bn - hb * Dm1);
      }
    }
  }
  for (int i = tid; i < N; i += nt) { gB[i] = sB[i]; gD[i] = sD[i]; }
}

// The FP32 auxiliary grid with one warp per source: every lane keeps 34
// consecutive cells of B and D in registers through the chunk, neighbours move
// by shuffles, and no block barrier is taken inside the time loop (the
// shared-memory form above, with six barriers a step, made the sources' grids
// cost as much as the batch they drive).  The grid's kTfsfAuxN cells are padded
// to kTfsfAuxPad = 32 x 34: the padding cells lie outside the grid, where every
// field is zero, so their damping factor is 0 and their E' is forced to 0.
// The update has the main kernels' form and FP32 weights (E' = S E*, H' = S H*;
// a + c = 1 and, for moving perturbation, c = 2 |cb| exactly), so the incident
// wave carries no drift of its own over long runs.  The damping factors, the
// same for every source, sit in shared memory.
constexpr int kAuxCPL = kTfsfAuxPad / 32;

template <int K> struct AuxCell { static constexpr int lane = K / kAuxCPL, c = K % kAuxCPL; };

__global__ void __launch_bounds__(128, 4) tfsf_aux_warp_kernel(const TfsfDev* __restrict__ tfs, int n_src,
                                                            float* __restrict__ aux, double* __restrict__ corr,
                                                            int chunk_stride, const long long* __restrict__ n_done,
                                                            int nsteps) {
  constexpr int N = kTfsfAuxN, P = kTfsfAuxPad, CPL = kAuxCPL;
  using Qm2 = AuxCell<kTfsfAuxQ - 2>;
  using Qm1 = AuxCell<kTfsfAuxQ - 1>;
  using Q0 = AuxCell<kTfsfAuxQ>;
  using Qp1 = AuxCell<kTfsfAuxQ + 1>;
  using Src = AuxCell<kTfsfAuxSrc>;
  __shared__ float sfB[P], sfD[P];
  for (int i = threadIdx.x; i < P; i += blockDim.x) {
    auto f = [](double x) {
      const double W = (double)kTfsfAuxW, right = (double)(N - 1) - W;
      double d = 0.0;
      if (x < W) d = (W - x) / W;
      else if (x > right) d = (x - right) / W;
      return (float)exp(-kTfsfAuxSigma * d * d);
    };
    sfB[i] = i < N ? f((double)i + 0.5) : 0.0f;
    sfD[i] = i < N ? f((double)i) : 0.0f;
  }
  __syncthreads();
  const int w = blockIdx.x * (blockDim.x >> 5) + (threadIdx.x >> 5);
  if (w >= n_src) return;                    // whole warps; no barrier follows
  const int lane = threadIdx.x & 31, k0 = lane * CPL;
  const TfsfDev tf = tfs[w];
  float* gB = aux + (size_t)w * 2 * P;
  float* gD = gB + P;
  float B[CPL], D[CPL];
#pragma unroll
  for (int c = 0; c < CPL; ++c) { B[c] = gB[k0 + c]; D[c] = gD[k0 + c]; }
  const float se = tf.se32, sm = tf.sm32, cb = tf.cb32, a = tf.a32, cc = tf.c32;
  const bool pos = tf.beta >= 0.0, first = lane == 0, last = lane == 31;
  const long long n0 = *n_done;
  double* out = corr + (size_t)w * chunk_stride * kTfsfCorr;
  for (int s = 0; s < nsteps; ++s) {
    const long long n = n0 + s + 1;
    // incident values before the step
    const float Bm2 = __shfl_sync(FULL, B[Qm2::c], Qm2::lane), Bm1 = __shfl_sync(FULL, B[Qm1::c], Qm1::lane);
    const float B0 = __shfl_sync(FULL, B[Q0::c], Q0::lane), Bp1 = __shfl_sync(FULL, B[Qp1::c], Qp1::lane);
    const float Dm1 = __shfl_sync(FULL, D[Qm1::c], Qm1::lane), D0 = __shfl_sync(FULL, D[Q0::c], Q0::lane);
    // E' = se D - cb (two B of the Table 1 average), then B^n (old B throughout)
    if (pos) {
      const float t1 = __shfl_up_sync(FULL, B[CPL - 1], 1), t2 = __shfl_up_sync(FULL, B[CPL - 2], 1);
      const float bl1 = first ? 0.0f : t1, bl2 = first ? 0.0f : t2;
      const float e0 = se * D[0] - cb * (bl1 + bl2);
      const float te = __shfl_down_sync(FULL, e0, 1);
      float en = last ? 0.0f : te;            // E' one cell to the right
#pragma unroll
      for (int c = CPL - 1; c >= 0; --c) {
        const float b1 = c >= 1 ? B[c - 1] : bl1;
        const float b2 = c >= 2 ? B[c - 2] : (c == 1 ? bl1 : bl2);
        const float ec = k0 + c < N ? se * D[c] - cb * (b1 + b2) : 0.0f;
        B[c] = (a * B[c] + (cc * b1 + (ec - en))) * sfB[k0 + c];
        en = ec;
      }
    } else {
      const float t1 = __shfl_down_sync(FULL, B[0], 1);
      const float br1 = last ? 0.0f : t1;
      const float e0 = se * D[0] - cb * (B[1] + B[0]);
      const float te = __shfl_down_sync(FULL, e0, 1);
      const float er = last ? 0.0f : te;
      float ec = e0;
#pragma unroll
      for (int c = 0; c < CPL; ++c) {
        const float b1 = c + 1 < CPL ? B[c + 1] : br1;
        const float b2 = c + 2 < CPL ? B[c + 2] : br1;          // used only for c + 2 == CPL
        const float en = c + 1 < CPL ? (k0 + c + 1 < N ? se * D[c + 1] - cb * (b2 + b1) : 0.0f) : er;
        B[c] = (a * B[c] + (cc * b1 + (ec - en))) * sfB[k0 + c];
        ec = en;
      }
    }
    // H' = sm B^n - cb (D_j + D_{j+1}) (D at level n-1/2), then D^{n+1/2} (old D throughout)
    {
      const float t1 = __shfl_down_sync(FULL, D[0], 1);
      const float dr = last ? 0.0f : t1;
      const float hlast = sm * B[CPL - 1] - cb * (D[CPL - 1] + dr);
      const float th = __shfl_up_sync(FULL, hlast, 1);
      const float hl = first ? 0.0f : th;
      if (pos) {
        const float t2 = __shfl_up_sync(FULL, D[CPL - 1], 1);
        const float dl = first ? 0.0f : t2;
        float hc = hlast;
#pragma unroll
        for (int c = CPL - 1; c >= 0; --c) {
          const float dp = c >= 1 ? D[c - 1] : dl;
          const float hp = c >= 1 ? sm * B[c - 1] - cb * (D[c - 1] + D[c]) : hl;
          D[c] = (a * D[c] + (cc * dp + (hp - hc))) * sfD[k0 + c];
          hc = hp;
        }
      } else {
        float hp = hl;
#pragma unroll
        for (int c = 0; c < CPL; ++c) {
          const float dn = c + 1 < CPL ? D[c + 1] : dr;
          const float hc = sm * B[c] - cb * (D[c] + dn);
          D[c] = (a * D[c] + (cc * dn + (hp - hc))) * sfD[k0 + c];
          hp = hc;
        }
      }
    }
    if (lane == Src::lane) {   // the source waveform in FP64, as for soft sources
      const double u = (double)(2 * n + 1) * tf.S * 0.5 - tf.t0;
      D[Src::c] += (float)(tf.amp * sin(tf.omega0 * u) * exp(-(u / tf.tau) * (u / tf.tau)));
    }
    const float Bn = __shfl_sync(FULL, B[Qm1::c], Qm1::lane);
    if (first) {
      const double se_ = se, sm_ = sm, cb_ = cb, uS = pos ? (double)cc : -(double)cc;   // uS = beta S
      double* c = out + (size_t)s * kTfsfCorr;
      if (pos) {
        c[0] = 0.0;
        c[1] = se_ * D0;
        c[2] = -cb_ * Bm2 + uS * Bm1;
        c[3] = -cb_ * Bm1;
        c[4] = -cb_ * D0;
        c[5] = (sm_ * Bn - cb_ * Dm1) + uS * Dm1;
      } else {
        c[0] = -cb_ * B0;
        c[1] = se_ * D0 - cb_ * Bp1 + uS * B0;
        c[2] = 0.0;
        c[3] = 0.0;
        c[4] = -cb_ * D0 + uS * D0;
        c[5] = sm_ * Bn - cb_ * Dm1;
      }
    }
  }
#pragma unroll
  for (int c = 0; c < CPL; ++c) { gB[k0 + c] = B[c]; gD[k0 + c] = D[c]; }
}

int tfsf_aux_launch(const TfsfDev* tf, int n, void* aux, bool fp64, double* corr, int chunk_stride,
                    const long long* n_done, int nsteps, cudaStream_t st) {
  if (n == 0 || nsteps == 0) return 0;
  if (fp64)
    tfsf_aux_kernel<double><<<n, kTfsfThreads, 0, st>>>(tf, (double*)aux, corr, chunk_stride, n_done, nsteps);
  else
    tfsf_aux_warp_kernel<<<(n + 3) / 4, 128, 0, st>>>(tf, n, (float*)aux, corr, chunk_stride, n_done, nsteps);
  return (int)cudaGetLastError();
}

}  // namespace gfdtd
