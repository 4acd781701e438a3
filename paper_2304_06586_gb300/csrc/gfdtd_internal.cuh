// gfdtd_internal.cuh -- device-side data layout shared by the kernels and the
// host API of the generalized-FDTD engine (not part of the public ABI).
#pragma once

#include <cuda_runtime.h>
#include <cuda_bf16.h>
#include <cuda_fp16.h>
#include <stdint.h>

namespace gfdtd {

// Instance flags.
enum : int {
  F_POS = 1,         // beta >= 0: Table 1 first column (Ba, dBa, dDa); else second column
  F_MATTER = 2,      // moving matter: per-node coupling beta_c (see gfdtd.h)
  F_LINEAR = 4,      // piecewise-linear profile (per-cell interpolation)
  F_MU_CONST = 8,    // H-side coefficients all equal (layers), or all mu knots equal (linear, not matter)
  F_EPS_CONST = 16,  // E-side coefficients all equal (layers), or all eps knots equal (linear, not matter)
};

// One instance of the batch, as the kernels see it.
struct InstDev {
  long long off;     // element offset of cell 0 in the field arrays (multiple of 32)
  long long dq;      // moving-frame displacement per half step, units of 2^-32 cell
  int nz;            // cells
  int nz_pad;        // nz rounded up to a multiple of 32
  int flags;
  int n;             // layers (LAYERS) or knots (LINEAR)
  int minw;          // LAYERS: smallest interior layer width in whole cells (node spacing of boundaries)
  int tab;           // first entry of this instance in the profile tables
  int src0, nsrc;    // sources: global indices [src0, src0 + nsrc)
  int prb0, nprb;    // probes: global indices [prb0, prb0 + nprb)
  double a;          // 1 - |beta| S   (upwind difference weight of the centre cell)
  double c;          // |beta| S       (weight of the upwind neighbour)
  double S;          // Courant number
  double inv_S;
  double beta;
  double cb;         // S beta / 2: coupling in the Table 1 averages (moving perturbation)
  float a32, c32, cb32;   // a, c, cb rounded to FP32 (the FP32-arithmetic kernels read these)
  float sm32;              // S / mu of the first layer or knot in FP32: the uniform value when F_MU_CONST
  int tf0, ntf;             // one-way sources of this instance: records tf0 .. tf0 + ntf - 1
  double abs_sigma;        // absorbing layers at both ends: strength at the outer end
  int abs_w;               // their width in cells (0: none)
  int pad2;
};
static_assert(sizeof(InstDev) % 16 == 0, "InstDev is copied by TMA in 16-byte units");

// Profile tables (concatenated over instances).
//   zq[tab + i]   : boundary (LAYERS, i < n-1) or knot (LINEAR, i < n) in 2^-32 cell
//   tabE[tab + i] : LAYERS: (S/eps_eff, S beta_c / 2) of layer i at integer nodes
//                   LINEAR: (eps, mu) at knot i
//   tabH[tab + i] : LAYERS: (S/mu_eff, S beta_c / 2) of layer i at half nodes
struct Tables {
  const long long* zq;
  const double2* tabE;
  const double2* tabH;
  const float2* tabE32;    // the same tables rounded to FP32 (for FP32 arithmetic)
  const float2* tabH32;
};

// Table access in the arithmetic type R (float or double).
template <typename R> struct TabOf;
template <> struct TabOf<float> {
  using V = float2;
  __device__ static const float2* get(const Tables& t, bool eside) { return eside ? t.tabE32 : t.tabH32; }
};
template <> struct TabOf<double> {
  using V = double2;
  __device__ static const double2* get(const Tables& t, bool eside) { return eside ? t.tabE : t.tabH; }
};

struct SrcDev {
  int inst;
  int node;
  double omega0, tau, t0, amp;
};

struct PrbDev {
  int inst;
  int node;
  int nbins;
  int bin0;          // first bin in the omega / accumulator arrays
};

// Tile geometry of the batched kernels.  A warp holds the window
// [base, base + 32 C) of an instance and advances it TB steps.  B'_j reads
// B_{j-2..j} and D_{j..j+1}, and D'_k reads D_{k-1..k+1} and B'_{k-1..k}
// (v >= 0; mirrored for v < 0), so after TB steps the cells still exact are
// [base + 2 TB + 1, base + 32 C - TB) for v >= 0 and [base + TB, base + 32 C - 2 TB)
// for v < 0.  The margin x0 - base and the output width are whole 16-byte
// vectors of V cells, so every copy of a tile is 16-byte aligned.
__host__ __device__ constexpr int tile_margin(int TB, bool pos, int V) {
  return ((pos ? 2 * TB + 1 : TB) + V - 1) / V * V;
}
__host__ __device__ constexpr int tile_width(int C, int TB, bool pos, int V) {
  return (32 * C - tile_margin(TB, pos, V) - (pos ? TB : 2 * TB)) / V * V;
}

// A tile of the fast kernel: where its input window starts in the field
// arrays and which sources and probes of its instance it holds (host-built).
struct FastTile {
  long long e;       // element offset of the first input cell: off + base
  int inst;          // instance
  int x0;            // first output cell
  unsigned smask;    // bit q: source src0 + q has its node in the tile's input window
  unsigned pmask;    // bit q: probe prb0 + q has its node among the tile's output cells
  int base;          // first cell of the window, x0 - tile_margin inside the domain
  int edge;          // bit 0: the window starts at cell 0; bit 1: it ends at or past nz,
                     // with (edge >> 8) cells of the window beyond nz
};
static_assert(sizeof(FastTile) == 32, "FastTile is copied by TMA in 16-byte units");

// Boundary tracker of one lane of a fast tile at the end of a launch.
struct TrackLane {
  long long dprev, dnext;    // zq + dq h - k0 2^32 of the boundaries around the lane's first cell
  long long dnext2;          // the same of the boundary after dnext (kernels that track two)
  float vL, vM, vR;          // sm se of the layers before, between and after dnext, dnext2 (FP32 kernels)
  int bnext;                 // index of the next boundary
  long long pad;
};
static_assert(sizeof(TrackLane) == 48, "TrackLane layout");
// The tracker state of a fast tile; n = the step count the state belongs to
// (-1: none).  Written at the end of each recording launch, read by the next.
struct TrackTile {
  long long n;
  long long pad;
  TrackLane lane[32];
};
static_assert(sizeof(TrackTile) % 16 == 0, "TrackTile is copied by TMA in 16-byte units");

// One-way (total-field / scattered-field) source: total field at nodes >= node.
// Its incident wave is computed in an auxiliary grid of the same scheme in
// the uniform background (the material at `node` at t = 0): kTfsfAuxN cells,
// graded absorbing layers of kTfsfAuxW cells and strength kTfsfAuxSigma at both
// ends of a 40-cell interior, a soft source with the given waveform at aux
// node kTfsfAuxSrc and the boundary at aux node kTfsfAuxQ.  (The layer width
// is the smallest power of two that reflects below 1e-6 of the incident wave
// in moving vacuum for |beta| <= 0.6.)  Each grid is stored as kTfsfAuxPad
// values of B then kTfsfAuxPad values of D, the cells past kTfsfAuxN held at
// zero, so that the FP32 kernel spreads a grid evenly over the 32 lanes of
// one warp.
struct TfsfDev {
  int inst;
  int node;
  double ie, im, hb;            // background 1/eps_m, 1/mu_m and beta_c / 2
  double beta, S;
  double omega0, tau, t0, amp;  // waveform of the auxiliary soft source
  float se32, sm32;             // FP32 weights of the background: S ie, S im,
  float cb32, a32, c32;         //   S hb, 1 - |beta| S, |beta| S (rounded as the main kernels' weights)
  float pad;
};
constexpr int kTfsfAuxN = 1064, kTfsfAuxW = 512, kTfsfAuxSrc = 520, kTfsfAuxQ = 532;
constexpr int kTfsfAuxPad = 1088;               // 32 lanes x 34 cells
static_assert(kTfsfAuxPad % 32 == 0 && kTfsfAuxPad >= kTfsfAuxN, "padded aux grid");
constexpr double kTfsfAuxSigma = 0.05;
constexpr int kTfsfCorr = 6;    // corrections per step: B at node-2 .. node+1, D at node-1 .. node

// Arguments of one time-block launch of the batched kernel.

template <typename T>
struct BlockArgs {
  const InstDev* inst;
  const int2* tiles;          // (instance, x0) of every tile
  int n_tiles;
  Tables tb;
  const SrcDev* srcs;
  const double* src_amp;      // [source][step in chunk]
  const PrbDev* prbs;
  double* samples;            // [probe][step in chunk]
  int chunk_stride;           // row length of src_amp and samples
  const T* Bin;
  const T* Din;
  T* Bout;
  T* Dout;
  const T* cBin;              // Kahan compensation of B and D (F32_KAHAN only)
  const T* cDin;
  T* cBout;
  T* cDout;
  const long long* n_done;    // steps completed at the start of the chunk (device)
  int s0;                     // first step of this launch within the chunk
  int nsteps;                 // steps in this launch (<= time block)
  int record;                 // nonzero: write probe samples
  int* err;                   // device status word: bit 0 = a bounded wait gave up
  const FastTile* ftiles;     // fast kernel: its tiles (n_tiles records, same order as `tiles`)
  TrackTile* track;           // fast kernel: tracker state per tile, kept between launches; NULL: not kept
  T* dseg;                    // general kernel: D after each step s goes to dseg + (s0 + s + 1) dseg_stride
  long long dseg_stride;      // (NULL: not recorded)
  const TfsfDev* tfsf;        // general kernel: one-way sources (instance i owns records
  int n_tfsf;                 //   tf0 .. tf0 + ntf - 1 of its InstDev; NULL or n_tfsf 0: none)
  const double* tf_corr;      // [source][step in chunk (chunk_stride)][kTfsfCorr] additive corrections
  int stall;                  // fast kernel, test hook: arm each tile barrier but start no copy,
                              //   so that every bounded wait runs out (0 in normal operation)
  int* queue;                 // general lists: uniform_kernel appends the tiles it does not take
  int* qcount;                //   (indices into `tiles`) and block_kernel takes them; qcount[0]:
                              //   entries, qcount[1]: blocks done (NULL: block_kernel takes every tile)
};

// Arguments of the plain kernel (one instance, one step).
template <typename T>
struct PlainArgs {
  InstDev I;                  // the instance's record (in the launch parameters)
  Tables tb;
  const SrcDev* srcs;
  const double* src_amp;      // source amplitudes of the chunk's steps (src_amp_launch)
  const PrbDev* prbs;
  double* samples;
  int chunk_stride;
  const long long* n_done;    // steps completed at the start of the chunk (device)
  const int* s_dev;           // step within the chunk (device): the step taken is *n_done + *s_dev + 1
  const T* Bin;
  const T* Din;
  T* Bout;
  T* Dout;
};
// Advances the plain path's step-within-chunk counter by one (after a step's launches).
int plain_tick_launch(int* s_dev, cudaStream_t st);
// gfdtd_plain_floor's launch: one instance's B and D read, output cells written back unchanged.
int plain_floor_launch(int elem_bytes, void* B, void* D, int nz, const int* s_dev, cudaStream_t st);

struct FoldArgs {
  const PrbDev* prbs;
  int n_prb;
  const double* samples;
  int chunk_stride;
  int nsteps;                 // samples per probe in this chunk
  const long long* n_done;    // steps completed at the start of the chunk
  const double* omega;        // all bins
  const int* bin_probe;       // probe of every bin
  int n_bins_total;
  double* acc_re;
  double* acc_im;
  double S;
};

// Adjoint (gfdtd_adjoint.cu).
struct SourceAdjArgs {
  int n_inst;
  const int* bin0;            // per instance: first bin of the loss band in the arrays below
  int nb;                     // bins per instance in the band
  const double* omega;        // all bins (global bin index)
  const double* Xre;          // loss-band DFT per global bin
  const double* Xim;
  long long n_first;          // first step of the segment
  int steps;
  double S;
  double* gn;                 // [step][inst]
};

// Time-blocked transpose: kAdjBlockSteps reverse steps per launch, a warp per
// tile of 32 x kAdjCells cells held in registers.  A tile's output range
// [x0, x0 + adj_width) sits in its window [x0 - adj_margin, x0 - adj_margin +
// 32 kAdjCells) with the margins one reverse step's stencil needs per step
// (cells j - 1 .. j + 3 for v >= 0, j - 2 .. j + 1 for v < 0).
constexpr int kAdjCells = 8;
constexpr int kAdjBlockSteps = 8;
__host__ __device__ constexpr int adj_margin(bool pos) { return pos ? kAdjBlockSteps : 2 * kAdjBlockSteps; }
__host__ __device__ constexpr int adj_width(bool pos) {
  return (32 * kAdjCells - adj_margin(pos) - (pos ? 3 * kAdjBlockSteps : kAdjBlockSteps)) / 4 * 4;
}
static_assert(adj_margin(true) % 4 == 0 && adj_margin(false) % 4 == 0, "windows start on 16-byte chunks");

struct AdjBlockArgs {
  const InstDev* inst;
  const int2* tiles;          // (instance, first output cell), adj_width(v >= 0) cells apart
  int n_tiles;
  Tables tb;
  const float* lBn;           // adjoint of B^{n_hi}, D^{n_hi+1/2}
  const float* lDn;
  float* lB;                  // adjoint of B^{n_hi-nsteps}, D^{n_hi-nsteps+1/2}
  float* lD;
  const float* dseg;          // D^{n+1/2} of the segment's step m (n = n_seg + m) at dseg + m * dseg_stride
  long long dseg_stride;
  long long n_seg;            // forward steps done at the segment's start
  int m_hi;                   // segment step of the first step transposed (n_hi = n_seg + m_hi)
  int nsteps;                 // steps transposed: m_hi, m_hi - 1, ..., m_hi - nsteps + 1 (<= kAdjBlockSteps)
  const int* probe_node;      // per instance (-1: none)
  const double* gn;           // dL/dF of segment step m for instance i at gn[(m - 1) n_inst + i]
  int n_inst;
  double* grad;               // dL/d(profile value), indexed by the instance's table offset
  int grad_copies;            // copies of grad, grad_stride apart: block b adds into copy b % copies
  long long grad_stride;
};
int adjoint_block_launch(const AdjBlockArgs& a, int grid, cudaStream_t st);
int adjoint_block_occupancy(int* blocks_per_sm);
// Advances the auxiliary grids of n one-way sources (FP64 or FP32 state, 2 kTfsfAuxPad
// values each) by nsteps steps from step *n_done and writes each step's corrections
// to corr ([source][chunk_stride][kTfsfCorr]).
int tfsf_aux_launch(const TfsfDev* tf, int n, void* aux, bool fp64, double* corr, int chunk_stride,
                    const long long* n_done, int nsteps, cudaStream_t st);
int sum_copies_launch(const double* copies, long long n_copies, long long stride, long long n, double* out,
                      cudaStream_t st);
int loss_source_launch(const SourceAdjArgs& a, cudaStream_t st);

// Kernel launchers (gfdtd_kernels.cu).
// variant: 0 general moving perturbation, 1 general moving matter, 2 fast interior tiles
// A tile shape is (C cells per lane, TB steps per time block, MB blocks per SM
// the fast kernel is register-limited to).
int block_launch(int prec, int variant, int C, int TB, int MB, const void* args, int grid, int block,
                 cudaStream_t st);
int block_occupancy(int prec, int variant, int C, int TB, int MB, int block, int* blocks_per_sm);
int block_shapes(int prec, int* C, int* TB, int* MB, int max);   // tile shapes built for a precision
int plain_launch(int prec, const void* args, int nz, cudaStream_t st);
int src_amp_launch(const SrcDev* srcs, int nsrc, double* amp, int stride, int nsteps,
                   const long long* n_done, double S, cudaStream_t st);
int fold_launch(const FoldArgs& a, cudaStream_t st);
// Runtime stability watchdog: block j of the scan covers the state elements
// [start, end) of instance inst (at most kWatchCells, 16-byte aligned).
struct WatchBlock {
  long long start, end;
  int inst, pad;
};
constexpr int kWatchCells = 8192;
// Merges, per instance, the largest |B| and |D| of the state (B, D in storage
// precision prec) into watch[inst] as the bits of its FP32 magnitude (NaNs above
// infinities above every finite value), by atomicMax.
int watch_launch(int prec, const WatchBlock* blocks, int n_blocks, const void* B, const void* D,
                 unsigned* watch, cudaStream_t st);
int advance_launch(long long* n_done, long long by, cudaStream_t st);
int convert_launch(int prec, int to_double, const void* src, void* dst, long long n, cudaStream_t st);
int capture_launch(int prec, int which, const InstDev* inst, int i, Tables tb, const void* B, const void* D,
                   long long z0, long long zs, long long m, long long n, int half, void* out, cudaStream_t st);
int derived_launch(int prec, int which, const InstDev* inst, int i, Tables tb, const void* B,
                   const void* D, double* out, int nz, long long n_done, cudaStream_t st);

}  // namespace gfdtd
