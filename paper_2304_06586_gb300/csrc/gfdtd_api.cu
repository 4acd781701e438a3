// gfdtd_api.cu -- host implementation of the C ABI declared in include/gfdtd.h.
//
// A context holds a batch of independent 1D instances.  All fields live in two
// ping-pong buffers per field (B, D) of padded per-instance segments; the
// moving-medium profiles live in small tables; time stepping is enqueued in
// chunks of at most kChunk steps, each chunk being [source amplitudes ->
// time-block launches -> DFT fold -> step counter advance], captured once
// per (chunk length, buffer parity) into a CUDA graph and replayed.
#include "../../include/gfdtd.h"
#include "gfdtd_block.cuh"
#include "gfdtd_medium.h"

#include <algorithm>
#include <cmath>
#include <complex>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <map>
#include <string>
#include <utility>
#include <vector>

namespace gfdtd {
int block_shapes(int prec, int* C, int* TB, int* MB, int max);
}

using namespace gfdtd;

namespace {

constexpr int kChunk = 1024;           // steps per chunk (probe/source buffers hold one chunk)
constexpr int kBlock = 128;            // threads per block of the batched kernel

gfdtd_alloc_fn g_alloc = nullptr;
gfdtd_free_fn g_free = nullptr;
void* g_user = nullptr;
std::string g_create_error;

int elem_bytes_of(gfdtd_prec p) {
  switch (p) {
    case GFDTD_F32: case GFDTD_F32_KAHAN: return 4;
    case GFDTD_BF16: case GFDTD_F16: return 2;
    case GFDTD_F64: return 8;
    default: return 0;
  }
}

struct Medium {
  gfdtd_kind kind = GFDTD_PERTURBATION;
  double beta = 0.0;
  gfdtd_interp interp = GFDTD_LAYERS;
  std::vector<double> z, eps{1.0}, mu{1.0};
  long long absorb_width = 0;     // absorbing layers at both ends (0: none)
  double absorb_sigma = 0.0;
};

struct Probe {
  int inst;
  long long node;
  std::vector<double> omega;
};

struct DevBuf {
  void* p = nullptr;
  size_t bytes = 0;
};

}  // namespace

struct gfdtd_ctx {
  int n_inst = 0;
  double S = 0.5;
  gfdtd_prec prec = GFDTD_F32;
  int eb = 4;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;   // internal stream used only for graph capture
  gfdtd_alloc_fn alloc = nullptr;
  gfdtd_free_fn free_fn = nullptr;
  void* user = nullptr;
  std::string err;

  std::vector<long long> nz, off;
  long long total = 0;                 // elements per field buffer
  std::vector<Medium> media;
  std::vector<std::vector<SrcDev>> sources;   // per instance
  std::vector<std::vector<TfsfDev>> tfsf;     // per instance: one-way sources (background filled by finalize)
  std::vector<Probe> probes;                  // in creation order
  std::vector<std::vector<int>> inst_probes;  // per instance: indices into `probes`

  // device state
  DevBuf B[2], D[2];
  DevBuf cB[2], cD[2];                  // Kahan compensation (F32_KAHAN only)
  int cur = 0;                          // buffer holding the current state
  DevBuf d_ndone;
  long long n_done = 0;
  DevBuf d_watch;                       // watchdog: one word per instance (see watch_launch)
  DevBuf d_watchblk;                    // the watchdog scan's blocks (WatchBlock)
  DevBuf d_plain_s;                     // plain path: step within the chunk (device counter)
  int n_watchblk = 0;
  int stall = 0;                        // test hook: fast-kernel tile copies are not started

  // device tables (rebuilt by finalize)
  bool dirty = true;
  DevBuf d_inst, d_zq, d_tabE, d_tabH, d_srcs, d_prbs, d_amp, d_samples, d_omega, d_binprb,
      d_acc_re, d_acc_im, d_tiles[3], d_tmp, d_tabE32, d_tabH32, d_ftiles, d_track;
  std::vector<InstDev> h_inst;
  std::vector<int> prb_global;          // probe creation index -> global (instance-sorted) index
  std::vector<int> prb_bin0;
  int n_src = 0, n_prb = 0, n_bins = 0;
  std::vector<double> acc_keep_re, acc_keep_im;   // accumulators per creation-order bin
  DevBuf d_tfsf, d_tfaux, d_tfcorr;     // one-way sources: records, auxiliary grids, corrections per chunk
  int n_tfsf = 0;

  // tiling
  int C = 0, TB = 0, MB = 0;            // chosen tile shape (0 = autotune)
  bool tuned = false;
  int n_tiles[3] = {0, 0, 0};           // [general perturbation, general matter, fast interior]
  long long valid_cells[3] = {0, 0, 0}; // exact output cells of each list's tiles per step
  int n_fast_damped = 0;                // the last ones of the fast list reach absorbing layers
  int grid[3] = {0, 0, 0};
  // uniform-tile queues of the general lists: counters (entries, warps done) of queues
  // 0, 1 (lists 0, 1 in gfdtd_step) and 2, 3 (lists 0, 2 in the adjoint's recomputation),
  // then the queues themselves
  DevBuf d_queue;
  int queue_off[4] = {0, 0, 0, 0};
  int ugrid[3] = {0, 0, 0};            // uniform_kernel grid per list (the context's precision)
  int ugrid_f32[3] = {0, 0, 0};        // the same in FP32 (the adjoint's recomputation)
  bool split = true;                   // general lists: uniform_kernel first (autotuned)
  int num_sms = 0;

  // adjoint work buffers (allocated on first use)
  // (two sets of the recomputation buffers: dseg, wB, adjn, amp2, one per segment in flight)
  DevBuf d_ckB, d_ckD, d_dseg[2], d_wB[2][2], d_amp2[2], d_lB[2], d_lD[2], d_grad, d_gn, d_adjn[2], d_Xre, d_Xim,
      d_bin0, d_pnode, d_acc0_re, d_acc0_im, d_adj_tiles;
  int n_adj_tiles = 0;
  int adj_grid = 1;

  // space-time capture: frames of one field of one instance every ts steps
  struct Capture {
    bool on = false;
    int inst = 0, which = 0, half = 0;
    long long z0 = 0, zs = 1, m = 0, ts = 0, max_frames = 0, frames = 0, dropped = 0, n_start = 0;
    DevBuf buf;
  } cap;

  // graphs keyed by (chunk length, parity)
  std::map<std::pair<int, int>, cudaGraphExec_t> graphs;
  long long launches = 0;
};

// ------------------------------------------------------------------ helpers

static gfdtd_status fail(gfdtd_ctx* c, gfdtd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (c) c->err = buf; else g_create_error = buf;
  return s;
}

#define CK(ctx, call)                                                                   \
  do {                                                                                  \
    cudaError_t e_ = (call);                                                            \
    if (e_ != cudaSuccess)                                                              \
      return fail(ctx, GFDTD_E_CUDA, "%s: %s (%s:%d)", #call, cudaGetErrorString(e_),    \
                  __FILE__, __LINE__);                                                  \
  } while (0)

#define CKI(ctx, expr)                                                                  \
  do {                                                                                  \
    int e_ = (expr);                                                                    \
    if (e_ != 0)                                                                        \
      return fail(ctx, GFDTD_E_CUDA, "%s: %s (%s:%d)", #expr,                            \
                  cudaGetErrorString((cudaError_t)e_), __FILE__, __LINE__);             \
  } while (0)

static gfdtd_status dalloc(gfdtd_ctx* c, DevBuf& b, size_t bytes) {
  if (b.p && b.bytes >= bytes && bytes > 0) return GFDTD_OK;
  if (b.p) {
    if (c->free_fn) c->free_fn(b.p, b.bytes, c->stream, c->user);
    else cudaFree(b.p);
    b.p = nullptr;
    b.bytes = 0;
  }
  if (bytes == 0) return GFDTD_OK;
  if (c->alloc) {
    b.p = c->alloc(bytes, c->stream, c->user);
    if (!b.p) return fail(c, GFDTD_E_OOM, "device allocation of %zu bytes failed", bytes);
  } else {
    cudaError_t e = cudaMalloc(&b.p, bytes);
    if (e != cudaSuccess) {
      b.p = nullptr;
      cudaGetLastError();
      return fail(c, GFDTD_E_OOM, "cudaMalloc(%zu): %s", bytes, cudaGetErrorString(e));
    }
  }
  b.bytes = bytes;
  return GFDTD_OK;
}

static void dfree(gfdtd_ctx* c, DevBuf& b) {
  if (!b.p) return;
  if (c->free_fn) c->free_fn(b.p, b.bytes, c->stream, c->user);
  else cudaFree(b.p);
  b.p = nullptr;
  b.bytes = 0;
}

template <typename V>
static gfdtd_status upload(gfdtd_ctx* c, DevBuf& b, const std::vector<V>& v) {
  const size_t bytes = std::max<size_t>(v.size() * sizeof(V), 16);
  gfdtd_status s = dalloc(c, b, bytes);
  if (s) return s;
  if (!v.empty()) CK(c, cudaMemcpyAsync(b.p, v.data(), v.size() * sizeof(V), cudaMemcpyHostToDevice, c->stream));
  return GFDTD_OK;
}

static void drop_graphs(gfdtd_ctx* c) {
  for (auto& kv : c->graphs) cudaGraphExecDestroy(kv.second);
  c->graphs.clear();
}

// Host von Neumann amplification (Sec. 5): 2x2 matrix of one Fourier mode.
static double max_zeta(double S, double beta, double ie, double im, double bc) {
  using cd = std::complex<double>;
  const cd I(0.0, 1.0);
  double worst = 0.0;
  const int nth = 4096;
  for (int i = 1; i <= nth; ++i) {
    const double th = M_PI * i / nth;
    cd bsum, adv;
    if (beta >= 0) { bsum = std::exp(-0.5 * I * th) + std::exp(-1.5 * I * th); adv = 1.0 - std::exp(-I * th); }
    else { bsum = std::exp(1.5 * I * th) + std::exp(0.5 * I * th); adv = std::exp(I * th) - 1.0; }
    const cd curl = 2.0 * I * std::sin(th / 2);
    const double avg = std::cos(th / 2);
    // E* = ie D - bc bsum/2 B;  B' = (1 - beta S adv) B - S curl E*
    const cd EsB = -bc * 0.5 * bsum, EsD = ie;
    const cd BB = 1.0 - beta * S * adv - S * curl * EsB, BD = -S * curl * EsD;
    // H* = im B' - bc avg D;  D' = (1 - beta S adv) D - S curl H*
    const cd HB = im * BB, HD = im * BD - bc * avg;
    const cd DB = -S * curl * HB, DD = 1.0 - beta * S * adv - S * curl * HD;
    const cd tr = BB + DD, det = BB * DD - BD * DB;
    const cd disc = std::sqrt(tr * tr - 4.0 * det);
    worst = std::max(worst, std::max(std::abs(0.5 * (tr + disc)), std::abs(0.5 * (tr - disc))));
  }
  return worst;
}

// Relative permittivity and permeability of a medium at moving coordinate xi
// (units of 2^-32 cell): a layers profile holds value i on [z_{i-1}, z_i), a
// linear one interpolates between knots and holds its end values beyond them.
static void medium_at(const Medium& m, long long xi, double& e, double& u) {
  const size_t n = m.eps.size();
  if (m.interp == GFDTD_LINEAR) {
    size_t j = 0;   // knots at or left of xi
    while (j < n && to_fixed(m.z[j]) <= xi) ++j;
    if (j == 0 || j == n) {
      const size_t k = j == 0 ? 0 : n - 1;
      e = m.eps[k];
      u = m.mu[k];
      return;
    }
    const long long z0 = to_fixed(m.z[j - 1]), z1 = to_fixed(m.z[j]);
    const double w = (double)(xi - z0) / (double)(z1 - z0);
    e = m.eps[j - 1] + w * (m.eps[j] - m.eps[j - 1]);
    u = m.mu[j - 1] + w * (m.mu[j] - m.mu[j - 1]);
    return;
  }
  size_t i = 0;     // boundaries at or left of xi
  while (i + 1 < n && to_fixed(m.z[i]) <= xi) ++i;
  e = m.eps[i];
  u = m.mu[i];
}

// ------------------------------------------------------------------ finalize

// Tiles of every instance, split by kernel variant: 0 general moving
// perturbation, 1 general moving matter, 2 fast interior tiles (see
// fast_kernel), with the fast kernel's tile records in `fast` (the order of
// out[2]).  Each list is ordered by the sign of v so that warps running at the
// same time execute the same code.
static gfdtd_status build_tiles(gfdtd_ctx* c, int C, int TB, std::vector<int2> out[3],
                                std::vector<FastTile>& fast) {
  std::vector<int2> part[3][2], pdamp[2];
  std::vector<FastTile> fpart[2], fdamp[2];   // fast tiles; those that reach an absorbing layer
  for (int v = 0; v < 3; ++v) c->valid_cells[v] = 0;
  for (int i = 0; i < c->n_inst; ++i) {
    const InstDev& d = c->h_inst[i];
    const bool pos = (d.flags & F_POS) != 0;
    const int W = tile_width(C, TB, pos, 16 / c->eb);
    const int L = tile_margin(TB, pos, 16 / c->eb);
    const bool matter = (d.flags & F_MATTER) != 0;
    const bool fast_ok = fast_eligible(d, C) && c->prec != GFDTD_F32_KAHAN;
    const long long nz = c->nz[i], V = 16 / c->eb, span = 32LL * C;
    for (long long x0 = 0; x0 < nz; x0 += W) {
      long long base = x0 - L;
      const bool left = base < 0, right = base + span > nz;
      // The fast kernel also takes a tile at one end of the domain: its window
      // is moved inside [0, nz) (the zero fields beyond the end are exact, so
      // no margin is needed on that side), rounded to whole vectors at the
      // right end.  Tiles at both ends, or whose window would not cover the
      // output range, stay with the general kernel.
      int edge = 0;
      bool fast_tile = fast_ok && !(left && right);
      // windows that hold a one-way source's correction cells run in the general kernel
      auto holds_tfsf = [&](long long b) {
        for (const TfsfDev& t : c->tfsf[i])
          if (t.node + 1 >= b && t.node - 2 < b + span) return true;
        return false;
      };
      if (holds_tfsf(base)) fast_tile = false;
      const bool damped = window_absorbs(d, base, span);
      if (fast_tile && left) {
        base = 0;
        edge = 1;
        if (span > nz) fast_tile = false;
      } else if (fast_tile && right) {
        base = (nz + V - 1) / V * V - span;
        edge = 2 | (int)((base + span - nz) << 8);
        // the two cells before nz must lie in the last lane's run (B_nz-1 + B_nz-2 term)
        if (base < 0 || base + L > x0 || base + span - nz > C - 2) fast_tile = false;
      }
      if (fast_tile && edge && holds_tfsf(base)) fast_tile = false;
      const int v = matter ? 1 : (fast_tile ? 2 : 0);
      (v == 2 && damped ? pdamp[pos ? 0 : 1] : part[v][pos ? 0 : 1]).push_back(make_int2(i, (int)x0));
      c->valid_cells[v] += std::min<long long>(W, nz - x0);
      if (v == 2) {
        FastTile f{};
        f.e = d.off + base;
        f.inst = i;
        f.x0 = (int)x0;
        f.base = (int)base;
        f.edge = edge;
        const std::vector<SrcDev>& src = c->sources[i];
        for (size_t q = 0; q < src.size() && q < 32; ++q)
          if (src[q].node >= base && src[q].node < base + 32LL * C) f.smask |= 1u << q;
        const std::vector<int>& prb = c->inst_probes[i];
        for (size_t q = 0; q < prb.size() && q < 32; ++q) {
          const long long node = c->probes[prb[q]].node;
          if (node >= x0 && node < x0 + W && node < c->nz[i]) f.pmask |= 1u << q;
        }
        (damped ? fdamp : fpart)[pos ? 0 : 1].push_back(f);
      }
    }
  }
  for (int v = 0; v < 3; ++v) {
    out[v] = part[v][0];
    out[v].insert(out[v].end(), part[v][1].begin(), part[v][1].end());
  }
  // the fast list ends with the tiles that reach an absorbing layer (their own launch)
  out[2].insert(out[2].end(), pdamp[0].begin(), pdamp[0].end());
  out[2].insert(out[2].end(), pdamp[1].begin(), pdamp[1].end());
  fast = fpart[0];
  fast.insert(fast.end(), fpart[1].begin(), fpart[1].end());
  for (int k = 0; k < 2; ++k) fast.insert(fast.end(), fdamp[k].begin(), fdamp[k].end());
  c->n_fast_damped = (int)(fdamp[0].size() + fdamp[1].size());
  if (out[0].size() + out[1].size() + out[2].size() > (size_t)INT32_MAX)
    return fail(c, GFDTD_E_ARG, "too many tiles");
  return GFDTD_OK;
}

static gfdtd_status set_tiles(gfdtd_ctx* c, int C, int TB, int MB) {
  std::vector<int2> t[3];
  std::vector<FastTile> ft;
  gfdtd_status s = build_tiles(c, C, TB, t, ft);
  if (s) return s;
  if ((s = upload(c, c->d_ftiles, ft))) return s;
  // per fast tile: the boundary trackers of its lanes, kept between launches (n = -1: none yet)
  const size_t track_bytes = std::max<size_t>(sizeof(TrackTile), ft.size() * sizeof(TrackTile));
  if ((s = dalloc(c, c->d_track, track_bytes))) return s;
  CK(c, cudaMemsetAsync(c->d_track.p, 0xff, track_bytes, c->stream));
  for (int k = 0; k < 3; ++k) {
    s = upload(c, c->d_tiles[k], t[k]);
    if (s) return s;
    c->n_tiles[k] = (int)t[k].size();
    int nb = 0;
    CKI(c, block_occupancy(c->prec, k, C, TB, MB, kBlock, &nb));
    nb = std::max(nb, 1);
    const int want = (c->n_tiles[k] + (kBlock / 32) - 1) / (kBlock / 32);
    c->grid[k] = std::max(1, std::min(c->num_sms * nb, want));
  }
  // uniform-tile queues (int entries): 16 counters, then lists 0, 1 and, for the
  // adjoint's recomputation, lists 0 and 2
  {
    const int sizes[4] = {c->n_tiles[0], c->n_tiles[1], c->n_tiles[0], c->n_tiles[2]};
    int off = 16;
    for (int q = 0; q < 4; ++q) {
      c->queue_off[q] = off;
      off += (sizes[q] + 3) / 4 * 4;
    }
    if ((s = dalloc(c, c->d_queue, (size_t)off * sizeof(int)))) return s;
    CK(c, cudaMemsetAsync(c->d_queue.p, 0, (size_t)off * sizeof(int), c->stream));
    for (int k = 0; k < 3; ++k) {
      c->ugrid[k] = c->ugrid_f32[k] = 0;
      const int want = std::max(1, (c->n_tiles[k] + (kBlock / 32) - 1) / (kBlock / 32));
      int nb = 0;
      if (c->prec != GFDTD_F32_KAHAN) {
        CKI(c, block_occupancy(c->prec, 4, C, TB, MB, kBlock, &nb));
        c->ugrid[k] = std::max(1, std::min(c->num_sms * std::max(nb, 1), want));
      }
      if (c->prec == GFDTD_F32 || c->prec == GFDTD_F32_KAHAN) {
        CKI(c, block_occupancy(GFDTD_F32, 4, C, TB, MB, kBlock, &nb));
        c->ugrid_f32[k] = std::max(1, std::min(c->num_sms * std::max(nb, 1), want));
      }
    }
  }
  c->C = C;
  c->TB = TB;
  c->MB = MB;
  drop_graphs(c);
  return GFDTD_OK;
}

// Queue q of the uniform-tile split (its counters and entries).
static int* queue_counts(gfdtd_ctx* c, int q) { return (int*)c->d_queue.p + 2 * q; }
static int* queue_entries(gfdtd_ctx* c, int q) { return (int*)c->d_queue.p + c->queue_off[q]; }

static gfdtd_status finalize(gfdtd_ctx* c) {
  if (!c->dirty) return GFDTD_OK;
  const double S = c->S;
  // preserve accumulators of existing probes across a rebuild
  if (c->n_bins > 0) {
    std::vector<double> re(c->n_bins), im(c->n_bins);
    CK(c, cudaMemcpyAsync(re.data(), c->d_acc_re.p, c->n_bins * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaMemcpyAsync(im.data(), c->d_acc_im.p, c->n_bins * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
    CK(c, cudaStreamSynchronize(c->stream));
    size_t pos = 0;
    c->acc_keep_re.assign(c->acc_keep_re.size(), 0.0);
    // old layout: global probe order; map back to creation order
    for (size_t p = 0; p < c->prb_global.size(); ++p) {
      const int g = c->prb_global[p];
      const int b0 = c->prb_bin0[g];
      const size_t nb = c->probes[p].omega.size();
      for (size_t j = 0; j < nb; ++j) {
        c->acc_keep_re[pos + j] = re[b0 + j];
        c->acc_keep_im[pos + j] = im[b0 + j];
      }
      pos += nb;
    }
  }
  std::vector<InstDev> inst(c->n_inst);
  std::vector<long long> zq;
  std::vector<double2> tabE, tabH;
  std::vector<float2> tabE32, tabH32;
  std::vector<SrcDev> srcs;
  std::vector<PrbDev> prbs;
  std::vector<double> omega, acc_re, acc_im;
  std::vector<int> binprb;
  c->prb_global.assign(c->probes.size(), 0);
  c->prb_bin0.clear();
  // creation-order bin offsets of each probe
  std::vector<size_t> keep_off(c->probes.size() + 1, 0);
  for (size_t p = 0; p < c->probes.size(); ++p) keep_off[p + 1] = keep_off[p] + c->probes[p].omega.size();
  int n_tf = 0;
  for (int i = 0; i < c->n_inst; ++i) {
    const Medium& m = c->media[i];
    InstDev& d = inst[i];
    d.tf0 = n_tf;
    d.ntf = (int)c->tfsf[i].size();
    n_tf += d.ntf;
    d.off = c->off[i];
    d.nz = (int)c->nz[i];
    d.nz_pad = (int)((c->nz[i] + 31) / 32 * 32);
    MediumSpec ms;
    ms.kind = (int)m.kind;
    ms.beta = m.beta;
    ms.interp = (int)m.interp;
    ms.n = (int)m.eps.size();
    ms.z = m.z.data();
    ms.eps = m.eps.data();
    ms.mu = m.mu.data();
    ms.absorb_width = m.absorb_width;
    ms.absorb_sigma = m.absorb_sigma;
    fill_instance(ms, S, d, zq, tabE, tabH, tabE32, tabH32);
    d.src0 = (int)srcs.size();
    d.nsrc = (int)c->sources[i].size();
    for (const SrcDev& s : c->sources[i]) srcs.push_back(s);
    d.prb0 = (int)prbs.size();
    d.nprb = (int)c->inst_probes[i].size();
    for (int p : c->inst_probes[i]) {
      const Probe& pr = c->probes[p];
      PrbDev pd;
      pd.inst = i;
      pd.node = (int)pr.node;
      pd.nbins = (int)pr.omega.size();
      pd.bin0 = (int)omega.size();
      c->prb_global[p] = (int)prbs.size();
      c->prb_bin0.push_back(pd.bin0);
      for (size_t j = 0; j < pr.omega.size(); ++j) {
        omega.push_back(pr.omega[j]);
        binprb.push_back((int)prbs.size());
        acc_re.push_back(c->acc_keep_re[keep_off[p] + j]);
        acc_im.push_back(c->acc_keep_im[keep_off[p] + j]);
      }
      prbs.push_back(pd);
    }
  }
  c->h_inst = inst;
  c->n_adj_tiles = 0;   // the adjoint's tiles follow the signs of v
  c->n_src = (int)srcs.size();
  c->n_prb = (int)prbs.size();
  c->n_bins = (int)omega.size();
  gfdtd_status s;
  if ((s = upload(c, c->d_inst, inst)) || (s = upload(c, c->d_zq, zq)) || (s = upload(c, c->d_tabE, tabE)) ||
      (s = upload(c, c->d_tabH, tabH)) || (s = upload(c, c->d_tabE32, tabE32)) ||
      (s = upload(c, c->d_tabH32, tabH32)) || (s = upload(c, c->d_srcs, srcs)) ||
      (s = upload(c, c->d_prbs, prbs)) || (s = upload(c, c->d_omega, omega)) ||
      (s = upload(c, c->d_binprb, binprb)) || (s = upload(c, c->d_acc_re, acc_re)) ||
      (s = upload(c, c->d_acc_im, acc_im)))
    return s;
  if (c->n_watchblk == 0) {   // the watchdog scan's blocks depend on the grid sizes only
    std::vector<WatchBlock> wb;
    for (int i = 0; i < c->n_inst; ++i) {
      const long long end = c->off[i] + (c->nz[i] + 31) / 32 * 32;
      for (long long b = c->off[i]; b < end; b += kWatchCells) {
        WatchBlock w{};
        w.start = b;
        w.end = std::min(end, b + kWatchCells);
        w.inst = i;
        wb.push_back(w);
      }
    }
    if ((s = upload(c, c->d_watchblk, wb))) return s;
    c->n_watchblk = (int)wb.size();
  }
  if ((s = dalloc(c, c->d_amp, std::max<size_t>(16, (size_t)c->n_src * kChunk * sizeof(double)))) ||
      (s = dalloc(c, c->d_samples, std::max<size_t>(16, (size_t)c->n_prb * kChunk * sizeof(double)))))
    return s;
  // one-way sources: background coefficients of the material at the boundary node at t = 0
  std::vector<TfsfDev> tfs;
  for (int i = 0; i < c->n_inst; ++i)
    for (TfsfDev t : c->tfsf[i]) {
      const Medium& m = c->media[i];
      double e, u;
      medium_at(m, (long long)t.node << 32, e, u);
      double ie, im, bc;
      medium_coefs((int)m.kind, m.beta, e, u, &ie, &im, &bc);
      t.ie = ie;
      t.im = im;
      t.hb = 0.5 * bc;
      t.beta = m.beta;
      t.S = S;
      t.se32 = (float)(S * ie);
      t.sm32 = (float)(S * im);
      t.cb32 = fp32_coupling(0.5 * S * bc);
      t.c32 = 2.0f * std::fabs(fp32_coupling(0.5 * S * m.beta));
      t.a32 = 1.0f - t.c32;
      tfs.push_back(t);
    }
  if ((s = upload(c, c->d_tfsf, tfs))) return s;
  if ((int)tfs.size() != c->n_tfsf) {
    // a new set of auxiliary grids starts from rest (the existing ones keep their state otherwise)
    const size_t aux_bytes = std::max<size_t>(16, tfs.size() * 2 * kTfsfAuxPad * sizeof(double));
    if ((s = dalloc(c, c->d_tfaux, aux_bytes)) ||
        (s = dalloc(c, c->d_tfcorr, std::max<size_t>(16, tfs.size() * kChunk * kTfsfCorr * sizeof(double)))))
      return s;
    CK(c, cudaMemsetAsync(c->d_tfaux.p, 0, aux_bytes, c->stream));
    c->n_tfsf = (int)tfs.size();
  }
  c->dirty = false;
  drop_graphs(c);
  if (c->C > 0) {
    s = set_tiles(c, c->C, c->TB, c->MB);
    if (s) return s;
  }
  return GFDTD_OK;
}

// ------------------------------------------------------------ enqueueing

static Tables tables_of(gfdtd_ctx* c) {
  Tables t;
  t.zq = (const long long*)c->d_zq.p;
  t.tabE = (const double2*)c->d_tabE.p;
  t.tabH = (const double2*)c->d_tabH.p;
  t.tabE32 = (const float2*)c->d_tabE32.p;
  t.tabH32 = (const float2*)c->d_tabH32.p;
  return t;
}

// Enqueue one time-block launch (both kinds) reading buffer `from`.
static gfdtd_status enqueue_block(gfdtd_ctx* c, cudaStream_t st, int from, int s0, int nsteps,
                                  bool record, bool sources, int only = -1, bool keep_track = false) {
  for (int k = 0; k < 3; ++k) {
    if (c->n_tiles[k] == 0 || (only >= 0 && k != only)) continue;
    // BlockArgs<T> has the same layout for every T (pointers), so fill the float version
    BlockArgs<float> a;
    a.inst = (const InstDev*)c->d_inst.p;
    a.tiles = (const int2*)c->d_tiles[k].p;
    a.n_tiles = c->n_tiles[k];
    a.tb = tables_of(c);
    a.srcs = (const SrcDev*)c->d_srcs.p;
    a.src_amp = sources ? (const double*)c->d_amp.p : nullptr;
    a.prbs = (const PrbDev*)c->d_prbs.p;
    a.samples = (double*)c->d_samples.p;
    a.chunk_stride = kChunk;
    a.Bin = (const float*)c->B[from].p;
    a.Din = (const float*)c->D[from].p;
    a.Bout = (float*)c->B[1 - from].p;
    a.Dout = (float*)c->D[1 - from].p;
    a.cBin = (const float*)c->cB[from].p;
    a.cDin = (const float*)c->cD[from].p;
    a.cBout = (float*)c->cB[1 - from].p;
    a.cDout = (float*)c->cD[1 - from].p;
    a.n_done = (const long long*)c->d_ndone.p;
    a.err = (int*)((char*)c->d_ndone.p + 8);
    a.ftiles = k == 2 ? (const FastTile*)c->d_ftiles.p : nullptr;
    a.track = (k == 2 && (record || keep_track)) ? (TrackTile*)c->d_track.p : nullptr;
    a.dseg = nullptr;
    a.dseg_stride = 0;
    a.tfsf = sources && c->n_tfsf > 0 ? (const TfsfDev*)c->d_tfsf.p : nullptr;
    a.n_tfsf = sources ? c->n_tfsf : 0;
    a.tf_corr = (const double*)c->d_tfcorr.p;
    a.s0 = s0;
    a.nsteps = nsteps;
    a.record = record ? 1 : 0;
    a.stall = c->stall;
    a.queue = nullptr;
    a.qcount = nullptr;
    if (k < 2 && c->split && c->prec != GFDTD_F32_KAHAN) {
      // tiles that see one material value over the launch step in uniform_kernel, the others
      // are queued for the general kernel
      a.queue = queue_entries(c, k);
      a.qcount = queue_counts(c, k);
      CKI(c, block_launch(c->prec, 4, c->C, c->TB, c->MB, &a, c->ugrid[k], kBlock, st));
      ++c->launches;
    }
    if (k == 2 && c->n_fast_damped > 0) {
      // the tiles that reach an absorbing layer, at the end of the list, get their own launch
      const int nd = c->n_fast_damped, nn = c->n_tiles[2] - nd;
      if (nn > 0) {
        a.n_tiles = nn;
        CKI(c, block_launch(c->prec, 2, c->C, c->TB, c->MB, &a, std::min(c->grid[2], (nn + 3) / 4), kBlock, st));
        ++c->launches;
      }
      BlockArgs<float> d = a;
      d.tiles = a.tiles + nn;
      d.ftiles = a.ftiles + nn;
      d.track = a.track ? a.track + nn : nullptr;
      d.n_tiles = nd;
      CKI(c, block_launch(c->prec, 3, c->C, c->TB, c->MB, &d, std::min(c->grid[2], (nd + 3) / 4), kBlock, st));
      ++c->launches;
      continue;
    }
    CKI(c, block_launch(c->prec, k, c->C, c->TB, c->MB, &a, c->grid[k], kBlock, st));
    ++c->launches;
  }
  return GFDTD_OK;
}

// End of a chunk: fold the probes' samples into their DFTs, scan the state
// (buffer state_buf) for the watchdog, advance the device step counter.
static gfdtd_status enqueue_fold_advance(gfdtd_ctx* c, cudaStream_t st, int nsteps, int state_buf) {
  if (c->n_watchblk > 0) {
    CKI(c, watch_launch(c->prec, (const WatchBlock*)c->d_watchblk.p, c->n_watchblk, c->B[state_buf].p,
                        c->D[state_buf].p, (unsigned*)c->d_watch.p, st));
    ++c->launches;
  }
  if (c->n_bins > 0) {
    FoldArgs f;
    f.prbs = (const PrbDev*)c->d_prbs.p;
    f.n_prb = c->n_prb;
    f.samples = (const double*)c->d_samples.p;
    f.chunk_stride = kChunk;
    f.nsteps = nsteps;
    f.n_done = (const long long*)c->d_ndone.p;
    f.omega = (const double*)c->d_omega.p;
    f.bin_probe = (const int*)c->d_binprb.p;
    f.n_bins_total = c->n_bins;
    f.acc_re = (double*)c->d_acc_re.p;
    f.acc_im = (double*)c->d_acc_im.p;
    f.S = c->S;
    CKI(c, fold_launch(f, st));
    ++c->launches;
  }
  CKI(c, advance_launch((long long*)c->d_ndone.p, nsteps, st));
  ++c->launches;
  return GFDTD_OK;
}

// One chunk of the batched path; returns the number of block launches (for parity).
static gfdtd_status enqueue_tfsf(gfdtd_ctx* c, cudaStream_t st, int nsteps) {
  if (c->n_tfsf > 0) {
    CKI(c, tfsf_aux_launch((const TfsfDev*)c->d_tfsf.p, c->n_tfsf, c->d_tfaux.p, c->prec == GFDTD_F64,
                           (double*)c->d_tfcorr.p, kChunk, (const long long*)c->d_ndone.p, nsteps, st));
    ++c->launches;
  }
  return GFDTD_OK;
}

static gfdtd_status enqueue_chunk(gfdtd_ctx* c, cudaStream_t st, int from, int nsteps, int* nlaunch) {
  if (c->n_src > 0) {
    CKI(c, src_amp_launch((const SrcDev*)c->d_srcs.p, c->n_src, (double*)c->d_amp.p, kChunk, nsteps,
                          (const long long*)c->d_ndone.p, c->S, st));
    ++c->launches;
  }
  gfdtd_status ts = enqueue_tfsf(c, st, nsteps);
  if (ts) return ts;
  int b = from, m = 0;
  for (int s0 = 0; s0 < nsteps; s0 += c->TB) {
    gfdtd_status s = enqueue_block(c, st, b, s0, std::min(c->TB, nsteps - s0), true, true);
    if (s) return s;
    b = 1 - b;
    ++m;
  }
  *nlaunch = m;
  return enqueue_fold_advance(c, st, nsteps, b);
}

static gfdtd_status run_chunk(gfdtd_ctx* c, int nsteps) {
  const auto key = std::make_pair(nsteps, c->cur);
  auto it = c->graphs.find(key);
  int m = (nsteps + c->TB - 1) / c->TB;
  if (it == c->graphs.end()) {
    cudaGraph_t g = nullptr;
    CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    const long long before = c->launches;
    gfdtd_status s = enqueue_chunk(c, c->cap_stream, c->cur, nsteps, &m);
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (s) { if (g) cudaGraphDestroy(g); return s; }
    CK(c, e);
    c->launches = before;   // counted at replay
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(c, e);
    it = c->graphs.emplace(key, ex).first;
  }
  CK(c, cudaGraphLaunch(it->second, c->stream));
  const int split = c->split && c->prec != GFDTD_F32_KAHAN ? 2 : 1;   // uniform_kernel + block_kernel per general list
  const int kinds = split * ((c->n_tiles[0] > 0) + (c->n_tiles[1] > 0)) + (c->n_tiles[2] > c->n_fast_damped) +
                    (c->n_fast_damped > 0);
  c->launches += (long long)m * kinds + (c->n_src > 0) + (c->n_tfsf > 0) + (c->n_bins > 0) +
                 (c->n_watchblk > 0) + 1;
  if (m & 1) c->cur = 1 - c->cur;
  c->n_done += nsteps;
  return GFDTD_OK;
}

// Time the candidate tile shapes on the actual batch (reads the current
// buffer, writes the other, records nothing) and keep the fastest.  The trial
// launches of a shape follow one another in time (s0 advances by a time block)
// so that, as in a real run, each finds the boundary trackers the previous one
// saved; set_tiles resets them for the shape finally kept.
// Device time per step of the current tiles over a few time blocks (reads the
// current buffer, writes the other, records nothing; the blocks follow one
// another in time so that each finds the boundary trackers the previous one saved).
static gfdtd_status time_blocks(gfdtd_ctx* c, int TB, cudaEvent_t e0, cudaEvent_t e1, double* per_step) {
  gfdtd_status s = enqueue_block(c, c->stream, c->cur, 0, TB, false, false, -1, true);
  if (s) return s;
  CK(c, cudaEventRecord(e0, c->stream));
  const int reps = 3;
  for (int r = 1; r <= reps; ++r) {
    s = enqueue_block(c, c->stream, c->cur, r * TB, TB, false, false, -1, true);
    if (s) return s;
  }
  CK(c, cudaEventRecord(e1, c->stream));
  CK(c, cudaEventSynchronize(e1));
  float ms = 0.f;
  CK(c, cudaEventElapsedTime(&ms, e0, e1));
  *per_step = (double)ms / (reps * TB);
  return GFDTD_OK;
}

static gfdtd_status autotune(gfdtd_ctx* c) {
  int Cs[16], TBs[16], MBs[16];
  const int n = block_shapes(c->prec, Cs, TBs, MBs, 16);
  if (n == 0) return fail(c, GFDTD_E_UNSUPPORTED, "no tile shape built for this precision");
  if (n == 1) return set_tiles(c, Cs[0], TBs[0], MBs[0]);
  cudaEvent_t e0, e1;
  CK(c, cudaEventCreate(&e0));
  CK(c, cudaEventCreate(&e1));
  // two passes over the candidates, each candidate keeping its faster pass, so
  // that a clock or cache transient during one timing does not decide alone
  // candidates: every shape, with and without the uniform-tile split of the general lists
  // where there are general tiles to split
  double per_step[16][2];
  bool general = false;
  for (int i = 0; i < n; ++i) per_step[i][0] = per_step[i][1] = 1e300;
  for (int pass = 0; pass < 2; ++pass) {
    for (int i = 0; i < n; ++i) {
      gfdtd_status s = set_tiles(c, Cs[i], TBs[i], MBs[i]);
      if (s) return s;
      general = (c->n_tiles[0] + c->n_tiles[1] > 0) && c->prec != GFDTD_F32_KAHAN;
      for (int sp = 0; sp < (general ? 2 : 1); ++sp) {
        c->split = sp == 0;
        double t = 0.0;
        s = time_blocks(c, TBs[i], e0, e1, &t);
        if (s) return s;
        per_step[i][sp] = std::min(per_step[i][sp], t);
      }
    }
  }
  int bi = 0, bs = 0;
  for (int i = 0; i < n; ++i)
    for (int sp = 0; sp < 2; ++sp)
      if (per_step[i][sp] < per_step[bi][bs]) { bi = i; bs = sp; }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  c->split = bs == 0;
  return set_tiles(c, Cs[bi], TBs[bi], MBs[bi]);
}

// Reads (after the stream is synchronised) the device status word that kernels
// set when a bounded wait gave up, and clears it.
static gfdtd_status device_status(gfdtd_ctx* c) {
  int err = 0;
  CK(c, cudaMemcpy(&err, (char*)c->d_ndone.p + 8, sizeof(int), cudaMemcpyDeviceToHost));
  if (err) {
    CK(c, cudaMemset((char*)c->d_ndone.p + 8, 0, sizeof(int)));
    return fail(c, GFDTD_E_TIMEOUT, "a kernel's bounded wait for its tile copy gave up (status %d)", err);
  }
  return GFDTD_OK;
}

static gfdtd_status check_inst(gfdtd_ctx* c, int inst) {
  if (!c) return GFDTD_E_ARG;
  if (inst < 0 || inst >= c->n_inst) return fail(c, GFDTD_E_ARG, "instance %d out of range", inst);
  return GFDTD_OK;
}


// Up to one time block of forward steps for the adjoint's segment recomputation:
// reads (Bin, dseg slice s0), writes Bout and D after every step into dseg
// slices s0 + 1 .. s0 + nsteps (the last one is also the block's D output).
// Every tile, the fast kernel's included, runs in the general FP32 kernel,
// whose per-step D store the reverse sweep needs.
constexpr int kGradCopies = 64;   // copies of the adjoint's gradient that its blocks spread atomics over

static gfdtd_status enqueue_segment_block(gfdtd_ctx* c, const void* Bin, void* Bout, char* dseg, size_t fb,
                                          const long long* n_done, int s0, int nsteps, const double* amp,
                                          cudaStream_t st) {
  for (int k : {0, 2}) {
    if (c->n_tiles[k] == 0) continue;
    BlockArgs<float> a{};
    a.inst = (const InstDev*)c->d_inst.p;
    a.tiles = (const int2*)c->d_tiles[k].p;
    a.n_tiles = c->n_tiles[k];
    a.tb = tables_of(c);
    a.srcs = (const SrcDev*)c->d_srcs.p;
    a.src_amp = c->n_src > 0 ? amp : nullptr;
    a.prbs = (const PrbDev*)c->d_prbs.p;
    a.samples = (double*)c->d_samples.p;
    a.chunk_stride = kChunk;
    a.Bin = (const float*)Bin;
    a.Din = (const float*)(dseg + (size_t)s0 * fb);
    a.Bout = (float*)Bout;
    a.Dout = (float*)(dseg + (size_t)(s0 + nsteps) * fb);
    a.n_done = n_done;
    a.err = (int*)((char*)c->d_ndone.p + 8);
    a.s0 = s0;
    a.nsteps = nsteps;
    a.record = 0;
    a.dseg = (float*)dseg;
    a.dseg_stride = (long long)(fb / sizeof(float));
    if (c->split) {
      // uniform tiles first (queue 2 or 3), the rest in the general kernel
      const int q = k == 0 ? 2 : 3;
      a.queue = queue_entries(c, q);
      a.qcount = queue_counts(c, q);
      CKI(c, block_launch(GFDTD_F32, 4, c->C, c->TB, c->MB, &a, c->ugrid_f32[k], kBlock, st));
      ++c->launches;
    }
    const int grid = std::min(c->grid[0] > 0 ? c->grid[0] : c->num_sms, (a.n_tiles + 3) / 4);
    CKI(c, block_launch(GFDTD_F32, 0, c->C, c->TB, c->MB, &a, std::max(grid, 1), kBlock, st));
    ++c->launches;
  }
  return GFDTD_OK;
}

extern "C" gfdtd_status gfdtd_adjoint(gfdtd_ctx* c, int64_t n_steps, int probe_id, int bin_lo,
                                      int bin_hi, double* loss, double* grad) {
  if (!c) return GFDTD_E_ARG;
  if (n_steps < 1 || !loss || !grad || bin_lo < 0 || bin_hi <= bin_lo)
    return fail(c, GFDTD_E_ARG, "need n_steps >= 1, 0 <= bin_lo < bin_hi, loss and grad");
  if (c->prec != GFDTD_F32 && c->prec != GFDTD_F32_KAHAN)
    return fail(c, GFDTD_E_UNSUPPORTED, "the adjoint is built for FP32 fields");
  for (int i = 0; i < c->n_inst; ++i) {
    if (c->media[i].kind != GFDTD_PERTURBATION)
      return fail(c, GFDTD_E_UNSUPPORTED, "the adjoint is built for moving perturbation");
    if (c->media[i].absorb_width > 0)
      return fail(c, GFDTD_E_UNSUPPORTED, "the adjoint has no absorbing layers");
    if (!c->tfsf[i].empty())
      return fail(c, GFDTD_E_UNSUPPORTED, "the adjoint covers soft sources only");
    if (probe_id < 0 || probe_id >= (int)c->inst_probes[i].size())
      return fail(c, GFDTD_E_ARG, "instance %d has no probe %d", i, probe_id);
    if ((int)c->probes[c->inst_probes[i][probe_id]].omega.size() < bin_hi)
      return fail(c, GFDTD_E_ARG, "instance %d: probe has fewer than %d bins", i, bin_hi);
  }
  gfdtd_status s = finalize(c);
  if (s) return s;
  if (c->C == 0 && (s = autotune(c))) return s;
  cudaStream_t st = c->stream;
  const long long N = n_steps;
  const long long K = (long long)std::ceil(std::sqrt((double)N));
  const long long nseg = (N + K - 1) / K;
  const size_t fb = (size_t)c->total * c->eb;          // bytes of one field buffer
  const size_t lb = (size_t)c->total * sizeof(float);
  const int ntab = (int)(c->d_tabE.bytes / sizeof(double2));
  if ((s = dalloc(c, c->d_ckB, fb * nseg)) || (s = dalloc(c, c->d_ckD, fb * nseg)) ||
      (s = dalloc(c, c->d_dseg[0], fb * (K + 1))) || (s = dalloc(c, c->d_dseg[1], fb * (K + 1))) ||
      (s = dalloc(c, c->d_wB[0][0], fb)) || (s = dalloc(c, c->d_wB[0][1], fb)) ||
      (s = dalloc(c, c->d_wB[1][0], fb)) || (s = dalloc(c, c->d_wB[1][1], fb)) ||
      (s = dalloc(c, c->d_amp2[0], std::max<size_t>(16, (size_t)c->n_src * kChunk * sizeof(double)))) ||
      (s = dalloc(c, c->d_amp2[1], std::max<size_t>(16, (size_t)c->n_src * kChunk * sizeof(double)))) ||
      (s = dalloc(c, c->d_lB[0], lb)) ||
      (s = dalloc(c, c->d_lB[1], lb)) || (s = dalloc(c, c->d_lD[0], lb)) ||
      (s = dalloc(c, c->d_lD[1], lb)) || (s = dalloc(c, c->d_grad, sizeof(double) * ntab * (kGradCopies + 1))) ||
      (s = dalloc(c, c->d_gn, sizeof(double) * K * c->n_inst)) || (s = dalloc(c, c->d_adjn[0], 16)) ||
      (s = dalloc(c, c->d_adjn[1], 16)) ||
      (s = dalloc(c, c->d_acc0_re, sizeof(double) * std::max(1, c->n_bins))) ||
      (s = dalloc(c, c->d_acc0_im, sizeof(double) * std::max(1, c->n_bins))))
    return s;
  // padding cells past nz are never written by the step kernels: keep them zero
  for (int b = 0; b < 2; ++b) {
    CK(c, cudaMemsetAsync(c->d_dseg[b].p, 0, fb * (K + 1), st));
    CK(c, cudaMemsetAsync(c->d_wB[b][0].p, 0, fb, st));
    CK(c, cudaMemsetAsync(c->d_wB[b][1].p, 0, fb, st));
  }
  if (c->n_adj_tiles == 0) {
    // tiles of the time-blocked transpose, those of instances with v >= 0 first (warps
    // running at the same time execute the same code)
    std::vector<int2> t;
    for (int side = 0; side < 2; ++side)
      for (int i = 0; i < c->n_inst; ++i) {
        const bool pos = (c->h_inst[i].flags & F_POS) != 0;
        if (pos != (side == 0)) continue;
        for (long long x0 = 0; x0 < c->nz[i]; x0 += adj_width(pos)) t.push_back(make_int2(i, (int)x0));
      }
    if ((s = upload(c, c->d_adj_tiles, t))) return s;
    c->n_adj_tiles = (int)t.size();
    int nb = 0;
    CKI(c, adjoint_block_occupancy(&nb));
    c->adj_grid = std::max(1, std::min(c->num_sms * std::max(nb, 1), (c->n_adj_tiles + 3) / 4));
  }
  // ---- forward with checkpoints at every segment start
  const long long n0 = c->n_done;
  CK(c, cudaMemcpyAsync(c->d_acc0_re.p, c->d_acc_re.p, sizeof(double) * c->n_bins, cudaMemcpyDeviceToDevice, st));
  CK(c, cudaMemcpyAsync(c->d_acc0_im.p, c->d_acc_im.p, sizeof(double) * c->n_bins, cudaMemcpyDeviceToDevice, st));
  for (long long sg = 0; sg < nseg; ++sg) {
    CK(c, cudaMemcpyAsync((char*)c->d_ckB.p + sg * fb, c->B[c->cur].p, fb, cudaMemcpyDeviceToDevice, st));
    CK(c, cudaMemcpyAsync((char*)c->d_ckD.p + sg * fb, c->D[c->cur].p, fb, cudaMemcpyDeviceToDevice, st));
    long long left = std::min(K, N - sg * K);
    while (left > 0) {
      const int ch = (int)std::min<long long>(left, kChunk);
      if ((s = run_chunk(c, ch))) return s;
      left -= ch;
    }
  }
  // ---- loss: L_i = sum over the band of |X_f|^2, X accumulated over these steps
  std::vector<double> re(c->n_bins), im(c->n_bins), re0(c->n_bins), im0(c->n_bins);
  CK(c, cudaMemcpyAsync(re.data(), c->d_acc_re.p, sizeof(double) * c->n_bins, cudaMemcpyDeviceToHost, st));
  CK(c, cudaMemcpyAsync(im.data(), c->d_acc_im.p, sizeof(double) * c->n_bins, cudaMemcpyDeviceToHost, st));
  CK(c, cudaMemcpyAsync(re0.data(), c->d_acc0_re.p, sizeof(double) * c->n_bins, cudaMemcpyDeviceToHost, st));
  CK(c, cudaMemcpyAsync(im0.data(), c->d_acc0_im.p, sizeof(double) * c->n_bins, cudaMemcpyDeviceToHost, st));
  CK(c, cudaStreamSynchronize(st));
  if ((s = device_status(c))) return s;
  std::vector<double> Xre(c->n_bins, 0.0), Xim(c->n_bins, 0.0);
  std::vector<int> bin0(c->n_inst), pnode(c->n_inst);
  for (int i = 0; i < c->n_inst; ++i) {
    const int p = c->inst_probes[i][probe_id];
    const int b0 = c->prb_bin0[c->prb_global[p]] + bin_lo;
    bin0[i] = b0;
    pnode[i] = (int)c->probes[p].node;
    double L = 0.0;
    for (int f = 0; f < bin_hi - bin_lo; ++f) {
      Xre[b0 + f] = re[b0 + f] - re0[b0 + f];
      Xim[b0 + f] = im[b0 + f] - im0[b0 + f];
      L += Xre[b0 + f] * Xre[b0 + f] + Xim[b0 + f] * Xim[b0 + f];
    }
    loss[i] = L;
  }
  if ((s = upload(c, c->d_Xre, Xre)) || (s = upload(c, c->d_Xim, Xim)) || (s = upload(c, c->d_bin0, bin0)) ||
      (s = upload(c, c->d_pnode, pnode)))
    return s;
  // ---- reverse sweep, segment by segment.  The forward recomputation of a
  // segment (general kernel, D after every step) runs on a second stream in
  // one of two buffer sets, one segment ahead of the reverse sweep, which
  // waits for it by an event; a set is refilled only after the reverse sweep
  // that read it has finished.
  CK(c, cudaMemsetAsync(c->d_lB[0].p, 0, lb, st));
  CK(c, cudaMemsetAsync(c->d_lD[0].p, 0, lb, st));
  CK(c, cudaMemsetAsync(c->d_grad.p, 0, sizeof(double) * ntab * (kGradCopies + 1), st));
  std::vector<long long> seg_n((size_t)nseg);          // steps done at each segment start
  for (long long sg = 0; sg < nseg; ++sg) seg_n[(size_t)sg] = n0 + sg * K;
  cudaStream_t st2 = nullptr;
  cudaEvent_t ev_start = nullptr, ev_rc[2] = {nullptr, nullptr}, ev_rv[2] = {nullptr, nullptr};
  struct Release {
    cudaStream_t& s2;
    cudaEvent_t& e0;
    cudaEvent_t* a;
    cudaEvent_t* b;
    ~Release() {
      if (s2) { cudaStreamSynchronize(s2); cudaStreamDestroy(s2); }
      for (cudaEvent_t e : {e0, a[0], a[1], b[0], b[1]}) if (e) cudaEventDestroy(e);
    }
  } release{st2, ev_start, ev_rc, ev_rv};
  CK(c, cudaStreamCreateWithFlags(&st2, cudaStreamNonBlocking));
  CK(c, cudaEventCreateWithFlags(&ev_start, cudaEventDisableTiming));
  for (int b = 0; b < 2; ++b) {
    CK(c, cudaEventCreateWithFlags(&ev_rc[b], cudaEventDisableTiming));
    CK(c, cudaEventCreateWithFlags(&ev_rv[b], cudaEventDisableTiming));
  }
  CK(c, cudaEventRecord(ev_start, st));               // checkpoints and buffer clears are done
  CK(c, cudaStreamWaitEvent(st2, ev_start, 0));
  auto recompute = [&](long long sg) -> gfdtd_status {
    const int bs = (int)(sg & 1);
    const int Ks = (int)std::min(K, N - sg * K);
    CK(c, cudaMemcpyAsync(c->d_adjn[bs].p, &seg_n[(size_t)sg], sizeof(long long), cudaMemcpyHostToDevice, st2));
    CK(c, cudaMemcpyAsync(c->d_wB[bs][0].p, (char*)c->d_ckB.p + sg * fb, fb, cudaMemcpyDeviceToDevice, st2));
    CK(c, cudaMemcpyAsync(c->d_dseg[bs].p, (char*)c->d_ckD.p + sg * fb, fb, cudaMemcpyDeviceToDevice, st2));
    if (c->n_src > 0) {
      CKI(c, src_amp_launch((const SrcDev*)c->d_srcs.p, c->n_src, (double*)c->d_amp2[bs].p, kChunk, Ks,
                            (const long long*)c->d_adjn[bs].p, c->S, st2));
      ++c->launches;
    }
    for (int m0 = 0, w = 0; m0 < Ks; m0 += c->TB, w ^= 1) {
      gfdtd_status r = enqueue_segment_block(c, c->d_wB[bs][w].p, c->d_wB[bs][w ^ 1].p, (char*)c->d_dseg[bs].p,
                                             fb, (const long long*)c->d_adjn[bs].p, m0, std::min(c->TB, Ks - m0),
                                             (const double*)c->d_amp2[bs].p, st2);
      if (r) return r;
    }
    CK(c, cudaEventRecord(ev_rc[bs], st2));
    return GFDTD_OK;
  };
  int lc = 0;
  auto reverse = [&](long long sg) -> gfdtd_status {
    const int bs = (int)(sg & 1);
    const long long ns = seg_n[(size_t)sg];
    const int Ks = (int)std::min(K, N - sg * K);
    CK(c, cudaStreamWaitEvent(st, ev_rc[bs], 0));
    SourceAdjArgs sa;
    sa.n_inst = c->n_inst;
    sa.bin0 = (const int*)c->d_bin0.p;
    sa.nb = bin_hi - bin_lo;
    sa.omega = (const double*)c->d_omega.p;
    sa.Xre = (const double*)c->d_Xre.p;
    sa.Xim = (const double*)c->d_Xim.p;
    sa.n_first = ns + 1;
    sa.steps = Ks;
    sa.S = c->S;
    sa.gn = (double*)c->d_gn.p;
    CKI(c, loss_source_launch(sa, st));
    ++c->launches;
    for (int m_hi = Ks; m_hi >= 1; m_hi -= kAdjBlockSteps) {
      AdjBlockArgs aa;
      aa.inst = (const InstDev*)c->d_inst.p;
      aa.tiles = (const int2*)c->d_adj_tiles.p;
      aa.n_tiles = c->n_adj_tiles;
      aa.tb = tables_of(c);
      aa.lBn = (const float*)c->d_lB[lc].p;
      aa.lDn = (const float*)c->d_lD[lc].p;
      aa.lB = (float*)c->d_lB[1 - lc].p;
      aa.lD = (float*)c->d_lD[1 - lc].p;
      aa.dseg = (const float*)c->d_dseg[bs].p;
      aa.dseg_stride = (long long)(fb / sizeof(float));
      aa.n_seg = ns;
      aa.m_hi = m_hi;
      aa.nsteps = std::min(kAdjBlockSteps, m_hi);
      aa.probe_node = (const int*)c->d_pnode.p;
      aa.gn = (const double*)c->d_gn.p;
      aa.n_inst = c->n_inst;
      aa.grad = (double*)c->d_grad.p;       // copies 0 .. kGradCopies-1; the sum goes after them
      aa.grad_copies = kGradCopies;
      aa.grad_stride = ntab;
      CKI(c, adjoint_block_launch(aa, c->adj_grid, st));
      ++c->launches;
      lc = 1 - lc;
    }
    CK(c, cudaEventRecord(ev_rv[bs], st));
    return GFDTD_OK;
  };
  if ((s = recompute(nseg - 1))) return s;
  if (nseg >= 2 && (s = recompute(nseg - 2))) return s;
  for (long long sg = nseg - 1; sg >= 0; --sg) {
    if ((s = reverse(sg))) return s;
    if (sg >= 2) {
      CK(c, cudaStreamWaitEvent(st2, ev_rv[sg & 1], 0));
      if ((s = recompute(sg - 2))) return s;
    }
  }
  std::vector<double> g(ntab);
  double* gsum = (double*)c->d_grad.p + (size_t)kGradCopies * ntab;
  CKI(c, sum_copies_launch((const double*)c->d_grad.p, kGradCopies, ntab, ntab, gsum, st));
  c->launches += 1;
  CK(c, cudaMemcpyAsync(g.data(), gsum, sizeof(double) * ntab, cudaMemcpyDeviceToHost, st));
  CK(c, cudaStreamSynchronize(st));
  size_t o = 0;
  for (int i = 0; i < c->n_inst; ++i) {
    const int nv = (int)c->media[i].eps.size();
    for (int j = 0; j < nv; ++j) grad[o + j] = g[c->h_inst[i].tab + j];
    o += nv;
  }
  return device_status(c);
}

// ================================================================== the ABI

extern "C" {

gfdtd_status gfdtd_set_allocator(gfdtd_alloc_fn alloc, gfdtd_free_fn free_fn, void* user) {
  if ((alloc == nullptr) != (free_fn == nullptr)) return GFDTD_E_ARG;
  g_alloc = alloc;
  g_free = free_fn;
  g_user = user;
  return GFDTD_OK;
}

gfdtd_status gfdtd_create(gfdtd_ctx** out, int n_inst, const int64_t* nz, double S,
                          gfdtd_prec prec, void* cuda_stream) {
  if (!out) return fail(nullptr, GFDTD_E_ARG, "out is NULL");
  *out = nullptr;
  if (n_inst < 1 || !nz) return fail(nullptr, GFDTD_E_ARG, "need n_inst >= 1 and nz");
  if (!(S > 0.0 && S <= 1.0)) return fail(nullptr, GFDTD_E_ARG, "S must be in (0, 1]");
  const int eb = elem_bytes_of(prec);
  if (eb == 0) return fail(nullptr, GFDTD_E_ARG, "unknown precision %d", (int)prec);
  for (int i = 0; i < n_inst; ++i)
    if (nz[i] < 1 || nz[i] > (1LL << 28))
      return fail(nullptr, GFDTD_E_ARG, "nz[%d] = %lld out of [1, 2^28]", i, (long long)nz[i]);
  gfdtd_ctx* c = new (std::nothrow) gfdtd_ctx;
  if (!c) return fail(nullptr, GFDTD_E_OOM, "host allocation failed");
  c->n_inst = n_inst;
  c->S = S;
  c->prec = prec;
  c->eb = eb;
  c->stream = (cudaStream_t)cuda_stream;
  c->alloc = g_alloc;
  c->free_fn = g_free;
  c->user = g_user;
  c->nz.assign(nz, nz + n_inst);
  c->off.resize(n_inst);
  long long o = 0;
  for (int i = 0; i < n_inst; ++i) {
    c->off[i] = o;
    o += (nz[i] + 31) / 32 * 32;
  }
  c->total = o + 32;   // one spare padded segment
  c->media.assign(n_inst, Medium());
  c->sources.assign(n_inst, {});
  c->tfsf.assign(n_inst, {});
  c->inst_probes.assign(n_inst, {});
  int dev = 0;
  gfdtd_status s = GFDTD_OK;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, dev);
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking);
  if (e != cudaSuccess) {
    g_create_error = std::string("CUDA initialisation failed: ") + cudaGetErrorString(e);
    delete c;
    return GFDTD_E_CUDA;
  }
  const size_t bytes = (size_t)c->total * eb;
  for (int k = 0; k < 2 && !s; ++k) {
    s = dalloc(c, c->B[k], bytes);
    if (!s) s = dalloc(c, c->D[k], bytes);
    if (!s && prec == GFDTD_F32_KAHAN) s = dalloc(c, c->cB[k], bytes);
    if (!s && prec == GFDTD_F32_KAHAN) s = dalloc(c, c->cD[k], bytes);
  }
  if (!s) s = dalloc(c, c->d_ndone, 16);
  if (!s) s = dalloc(c, c->d_watch, sizeof(unsigned) * (size_t)n_inst);
  if (!s) {
    cudaMemsetAsync(c->d_watch.p, 0, sizeof(unsigned) * (size_t)n_inst, c->stream);
    for (int k = 0; k < 2; ++k) {
      cudaMemsetAsync(c->B[k].p, 0, bytes, c->stream);
      cudaMemsetAsync(c->D[k].p, 0, bytes, c->stream);
      if (c->cB[k].p) cudaMemsetAsync(c->cB[k].p, 0, bytes, c->stream);
      if (c->cD[k].p) cudaMemsetAsync(c->cD[k].p, 0, bytes, c->stream);
    }
    cudaMemsetAsync(c->d_ndone.p, 0, 16, c->stream);
    if (cudaGetLastError() != cudaSuccess) s = fail(c, GFDTD_E_CUDA, "memset failed");
  }
  if (s) {
    g_create_error = c->err;
    gfdtd_destroy(c);
    return s;
  }
  *out = c;
  return GFDTD_OK;
}

gfdtd_status gfdtd_set_medium(gfdtd_ctx* c, int inst, gfdtd_kind kind, double beta,
                              gfdtd_interp interp, int n, const double* z, const double* eps_r,
                              const double* mu_r, int allow_unstable) {
  gfdtd_status s = check_inst(c, inst);
  if (s) return s;
  if (kind != GFDTD_PERTURBATION && kind != GFDTD_MATTER) return fail(c, GFDTD_E_ARG, "bad kind");
  if (interp != GFDTD_LAYERS && interp != GFDTD_LINEAR) return fail(c, GFDTD_E_ARG, "bad interp");
  if (!(beta > -1.0 && beta < 1.0)) return fail(c, GFDTD_E_ARG, "beta must be in (-1, 1)");
  if (std::fabs(beta) * c->S >= 1.0) return fail(c, GFDTD_E_ARG, "|beta| S must be < 1");
  if (n < 1 || (interp == GFDTD_LINEAR && n < 2) || !eps_r || !mu_r)
    return fail(c, GFDTD_E_ARG, "need n >= 1 values (n >= 2 knots for LINEAR)");
  const int nz_pos = interp == GFDTD_LAYERS ? n - 1 : n;
  if (nz_pos > 0 && !z) return fail(c, GFDTD_E_ARG, "z is NULL");
  for (int i = 0; i < n; ++i)
    if (!(eps_r[i] > 0.0) || !(mu_r[i] > 0.0)) return fail(c, GFDTD_E_ARG, "eps and mu must be > 0");
  for (int i = 0; i < nz_pos; ++i) {
    if (!std::isfinite(z[i]) || std::fabs(z[i]) > 1e9) return fail(c, GFDTD_E_ARG, "bad position");
    if (i > 0 && !(z[i] > z[i - 1])) return fail(c, GFDTD_E_ARG, "positions must increase");
  }
  if (!allow_unstable) {
    for (int i = 0; i < n; ++i) {
      bool seen = false;   // each distinct (eps, mu) pair is analysed once
      for (int j = 0; j < i && !seen; ++j) seen = eps_r[j] == eps_r[i] && mu_r[j] == mu_r[i];
      if (seen) continue;
      double ie, im, bc;
      medium_coefs((int)kind, beta, eps_r[i], mu_r[i], &ie, &im, &bc);
      const double g = max_zeta(c->S, beta, ie, im, bc);
      if (g > 1.0 + 1e-9)
        return fail(c, GFDTD_E_UNSTABLE, "eps=%g mu=%g beta=%g: max|zeta| = %.9f > 1 (n|beta| > 1)",
                    eps_r[i], mu_r[i], beta, g);
    }
  }
  Medium& m = c->media[inst];
  m.kind = kind;
  m.beta = beta;
  m.interp = interp;
  m.z.assign(z ? z : eps_r, (z ? z : eps_r) + (z ? nz_pos : 0));
  m.eps.assign(eps_r, eps_r + n);
  m.mu.assign(mu_r, mu_r + n);
  c->dirty = true;
  return GFDTD_OK;
}

gfdtd_status gfdtd_set_absorber(gfdtd_ctx* c, int inst, int64_t width, double sigma) {
  gfdtd_status s = check_inst(c, inst);
  if (s) return s;
  if (width < 0 || 2 * width >= c->nz[inst] || !(sigma >= 0.0) || !std::isfinite(sigma))
    return fail(c, GFDTD_E_ARG, "need 0 <= width, 2 width < nz and a finite sigma >= 0");
  c->media[inst].absorb_width = width;
  c->media[inst].absorb_sigma = sigma;
  c->dirty = true;
  return GFDTD_OK;
}

gfdtd_status gfdtd_add_source(gfdtd_ctx* c, int inst, int64_t node, double omega0, double tau,
                              double t0, double amp) {
  gfdtd_status s = check_inst(c, inst);
  if (s) return s;
  if (node < 0 || node >= c->nz[inst]) return fail(c, GFDTD_E_ARG, "source node out of range");
  if (!(tau > 0.0) || !std::isfinite(omega0) || !std::isfinite(t0) || !std::isfinite(amp))
    return fail(c, GFDTD_E_ARG, "bad source parameters");
  if (c->sources[inst].size() >= 32) return fail(c, GFDTD_E_ARG, "at most 32 sources per instance");
  SrcDev d;
  d.inst = inst;
  d.node = (int)node;
  d.omega0 = omega0;
  d.tau = tau;
  d.t0 = t0;
  d.amp = amp;
  c->sources[inst].push_back(d);
  c->dirty = true;
  return GFDTD_OK;
}

gfdtd_status gfdtd_add_tfsf(gfdtd_ctx* c, int inst, int64_t node, double omega0, double tau, double t0,
                            double amp) {
  gfdtd_status s = check_inst(c, inst);
  if (s) return s;
  if (node < 0 || node >= c->nz[inst]) return fail(c, GFDTD_E_ARG, "one-way source node out of range");
  if (!(tau > 0.0) || !std::isfinite(omega0) || !std::isfinite(t0) || !std::isfinite(amp))
    return fail(c, GFDTD_E_ARG, "bad source parameters");
  if (c->tfsf[inst].size() >= 4) return fail(c, GFDTD_E_ARG, "at most 4 one-way sources per instance");
  TfsfDev t{};
  t.inst = inst;
  t.node = (int)node;
  t.omega0 = omega0;
  t.tau = tau;
  t.t0 = t0;
  t.amp = amp;
  c->tfsf[inst].push_back(t);
  c->dirty = true;
  return GFDTD_OK;
}

gfdtd_status gfdtd_add_probe(gfdtd_ctx* c, int inst, int64_t node, int n_bins, const double* omega,
                             int* probe_id) {
  gfdtd_status s = check_inst(c, inst);
  if (s) return s;
  if (node < 0 || node >= c->nz[inst]) return fail(c, GFDTD_E_ARG, "probe node out of range");
  if (n_bins < 1 || !omega || !probe_id) return fail(c, GFDTD_E_ARG, "need n_bins >= 1, omega, probe_id");
  if (c->inst_probes[inst].size() >= 32) return fail(c, GFDTD_E_ARG, "at most 32 probes per instance");
  Probe p;
  p.inst = inst;
  p.node = node;
  p.omega.assign(omega, omega + n_bins);
  c->probes.push_back(p);
  c->inst_probes[inst].push_back((int)c->probes.size() - 1);
  c->acc_keep_re.resize(c->acc_keep_re.size() + n_bins, 0.0);
  c->acc_keep_im.resize(c->acc_keep_im.size() + n_bins, 0.0);
  *probe_id = (int)c->inst_probes[inst].size() - 1;
  c->dirty = true;
  return GFDTD_OK;
}

gfdtd_status gfdtd_step(gfdtd_ctx* c, int64_t n_steps) {
  if (!c) return GFDTD_E_ARG;
  if (n_steps < 0) return fail(c, GFDTD_E_ARG, "n_steps < 0");
  gfdtd_status s = finalize(c);
  if (s) return s;
  if (c->C == 0) {
    s = autotune(c);
    if (s) return s;
  }
  while (n_steps > 0) {
    int ch = (int)std::min<int64_t>(n_steps, kChunk);
    if (c->cap.on)   // end the chunk at the next frame
      ch = (int)std::min<long long>(ch, c->cap.ts - (c->n_done - c->cap.n_start) % c->cap.ts);
    s = run_chunk(c, ch);
    if (s) return s;
    n_steps -= ch;
    if (c->cap.on && (c->n_done - c->cap.n_start) % c->cap.ts == 0) {
      gfdtd_ctx::Capture& k = c->cap;
      if (k.frames < k.max_frames) {
        char* dst = (char*)k.buf.p + (size_t)(k.frames * k.m) * (k.half ? 2 : 4);
        CKI(c, capture_launch(c->prec, k.which, (const InstDev*)c->d_inst.p, k.inst, tables_of(c),
                              c->B[c->cur].p, c->D[c->cur].p, k.z0, k.zs, k.m, c->n_done, k.half, dst,
                              c->stream));
        ++c->launches;
        ++k.frames;
      } else {
        ++k.dropped;
      }
    }
  }
  return GFDTD_OK;
}

gfdtd_status gfdtd_set_capture(gfdtd_ctx* c, int inst, gfdtd_field which, int64_t z0, int64_t z1,
                               int64_t z_stride, int64_t t_stride, int64_t max_frames, int half) {
  if (!c) return GFDTD_E_ARG;
  if (t_stride == 0) {
    c->cap.on = false;
    return GFDTD_OK;
  }
  gfdtd_status s = check_inst(c, inst);
  if (s) return s;
  if (which < GFDTD_FIELD_D || which > GFDTD_FIELD_ESTAR) return fail(c, GFDTD_E_ARG, "bad field");
  if (which == GFDTD_FIELD_H && c->media[inst].kind == GFDTD_MATTER)
    return fail(c, GFDTD_E_UNSUPPORTED, "H is not available for moving matter");
  if (z0 < 0 || z1 > c->nz[inst] || z0 >= z1 || z_stride < 1 || t_stride < 1 || max_frames < 1 ||
      (half != 0 && half != 1))
    return fail(c, GFDTD_E_ARG, "need 0 <= z0 < z1 <= nz, strides >= 1, max_frames >= 1, half 0 or 1");
  const long long m = (z1 - z0 + z_stride - 1) / z_stride;
  if ((s = dalloc(c, c->cap.buf, (size_t)(max_frames * m) * (half ? 2 : 4)))) return s;
  gfdtd_ctx::Capture& k = c->cap;
  k.on = true;
  k.inst = inst;
  k.which = (int)which;
  k.half = half;
  k.z0 = z0;
  k.zs = z_stride;
  k.m = m;
  k.ts = t_stride;
  k.max_frames = max_frames;
  k.frames = 0;
  k.dropped = 0;
  k.n_start = c->n_done;
  return GFDTD_OK;
}

gfdtd_status gfdtd_capture_info(const gfdtd_ctx* c, int64_t* frames, int64_t* cells_per_frame,
                                int64_t* dropped) {
  if (!c || !frames || !cells_per_frame || !dropped) return GFDTD_E_ARG;
  *frames = c->cap.frames;
  *cells_per_frame = c->cap.m;
  *dropped = c->cap.dropped;
  return GFDTD_OK;
}

gfdtd_status gfdtd_read_capture(gfdtd_ctx* c, double* host_dst, int64_t n) {
  if (!c) return GFDTD_E_ARG;
  const long long have = c->cap.frames * c->cap.m;
  if (!host_dst || n != have) return fail(c, GFDTD_E_ARG, "n must equal frames x cells_per_frame (%lld)", have);
  if (n == 0) return GFDTD_OK;
  gfdtd_status s = dalloc(c, c->d_tmp, (size_t)n * sizeof(double));
  if (s) return s;
  // frames are stored in FP32 or FP16: widen with the converters of those storage types
  CKI(c, convert_launch(c->cap.half ? GFDTD_F16 : GFDTD_F32, 1, c->cap.buf.p, c->d_tmp.p, n, c->stream));
  CK(c, cudaMemcpyAsync(host_dst, c->d_tmp.p, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return device_status(c);
}

gfdtd_status gfdtd_profile_kernels(gfdtd_ctx* c, int64_t n_steps, gfdtd_kernel_times* out) {
  if (!c) return GFDTD_E_ARG;
  if (!out) return fail(c, GFDTD_E_ARG, "out is NULL");
  if (n_steps < 0) return fail(c, GFDTD_E_ARG, "n_steps < 0");
  gfdtd_status s = finalize(c);
  if (s) return s;
  if (c->C == 0) {
    s = autotune(c);
    if (s) return s;
  }
  struct Mark { int k; int nsteps; cudaEvent_t e0, e1; };
  std::vector<Mark> marks;
  auto release = [&]() {
    for (Mark& m : marks) { cudaEventDestroy(m.e0); cudaEventDestroy(m.e1); }
    marks.clear();
  };
  gfdtd_kernel_times r;
  std::memset(&r, 0, sizeof r);
  while (n_steps > 0 && s == GFDTD_OK) {
    const int ch = (int)std::min<int64_t>(n_steps, kChunk);
    if (c->n_src > 0) {
      if (src_amp_launch((const SrcDev*)c->d_srcs.p, c->n_src, (double*)c->d_amp.p, kChunk, ch,
                         (const long long*)c->d_ndone.p, c->S, c->stream) != 0) {
        s = fail(c, GFDTD_E_CUDA, "source amplitude launch failed");
        break;
      }
      ++c->launches;
    }
    if (s == GFDTD_OK) s = enqueue_tfsf(c, c->stream, ch);
    int b = c->cur, m = 0;
    for (int s0 = 0; s0 < ch && s == GFDTD_OK; s0 += c->TB) {
      const int nsteps = std::min(c->TB, ch - s0);
      for (int k = 0; k < 3 && s == GFDTD_OK; ++k) {
        if (c->n_tiles[k] == 0) continue;
        Mark mk{k, nsteps, nullptr, nullptr};
        if (cudaEventCreate(&mk.e0) != cudaSuccess || cudaEventCreate(&mk.e1) != cudaSuccess) {
          if (mk.e0) cudaEventDestroy(mk.e0);
          s = fail(c, GFDTD_E_CUDA, "cudaEventCreate failed");
          break;
        }
        marks.push_back(mk);
        if (cudaEventRecord(mk.e0, c->stream) != cudaSuccess) { s = fail(c, GFDTD_E_CUDA, "event record failed"); break; }
        s = enqueue_block(c, c->stream, b, s0, nsteps, true, true, k);
        if (s) break;
        if (cudaEventRecord(mk.e1, c->stream) != cudaSuccess) { s = fail(c, GFDTD_E_CUDA, "event record failed"); break; }
      }
      b = 1 - b;
      ++m;
    }
    if (s) break;
    s = enqueue_fold_advance(c, c->stream, ch, b);
    if (s) break;
    if (m & 1) c->cur = 1 - c->cur;
    c->n_done += ch;
    n_steps -= ch;
  }
  if (s == GFDTD_OK && cudaStreamSynchronize(c->stream) != cudaSuccess)
    s = fail(c, GFDTD_E_CUDA, "%s", cudaGetErrorString(cudaGetLastError()));
  if (s == GFDTD_OK) {
    for (const Mark& mk : marks) {
      float ms = 0.0f;
      if (cudaEventElapsedTime(&ms, mk.e0, mk.e1) != cudaSuccess) {
        s = fail(c, GFDTD_E_CUDA, "cudaEventElapsedTime failed");
        break;
      }
      r.launches[mk.k] += 1;
      r.ms[mk.k] += ms;
      r.cell_updates[mk.k] += c->valid_cells[mk.k] * mk.nsteps;
    }
  }
  release();
  if (s == GFDTD_OK) s = device_status(c);
  if (s == GFDTD_OK) *out = r;
  return s;
}

gfdtd_status gfdtd_step_plain(gfdtd_ctx* c, int64_t n_steps) {
  if (!c) return GFDTD_E_ARG;
  if (c->prec == GFDTD_F32_KAHAN)
    return fail(c, GFDTD_E_UNSUPPORTED, "the plain kernel has no compensated tier");
  if (n_steps < 0) return fail(c, GFDTD_E_ARG, "n_steps < 0");
  gfdtd_status s = finalize(c);
  if (s) return s;
  if (c->n_tfsf > 0) return fail(c, GFDTD_E_UNSUPPORTED, "one-way sources run in gfdtd_step only");
  // One step = one launch per instance, in instance order on the stream, then a
  // tick of the device step counter; the launches of a step read the step from
  // device memory, so one captured CUDA graph per buffer parity replays every
  // step (the launches stay one instance and one step each).
  if (!c->d_plain_s.p) {
    s = dalloc(c, c->d_plain_s, 16);
    if (s) return s;
  }
  while (n_steps > 0) {
    const int ch = (int)std::min<int64_t>(n_steps, kChunk);
    CK(c, cudaMemsetAsync(c->d_plain_s.p, 0, sizeof(int), c->stream));
    if (c->n_src > 0) {
      CKI(c, src_amp_launch((const SrcDev*)c->d_srcs.p, c->n_src, (double*)c->d_amp.p, kChunk, ch,
                            (const long long*)c->d_ndone.p, c->S, c->stream));
      ++c->launches;
    }
    for (int st = 0; st < ch; ++st) {
      const auto key = std::make_pair(-1, c->cur);
      auto it = c->graphs.find(key);
      if (it == c->graphs.end()) {
        cudaGraph_t g = nullptr;
        CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
        gfdtd_status cs = GFDTD_OK;
        for (int i = 0; i < c->n_inst && !cs; ++i) {
          PlainArgs<float> a;
          a.I = c->h_inst[i];
          a.tb = tables_of(c);
          a.srcs = (const SrcDev*)c->d_srcs.p;
          a.src_amp = (const double*)c->d_amp.p;
          a.prbs = (const PrbDev*)c->d_prbs.p;
          a.samples = (double*)c->d_samples.p;
          a.chunk_stride = kChunk;
          a.n_done = (const long long*)c->d_ndone.p;
          a.s_dev = (const int*)c->d_plain_s.p;
          a.Bin = (const float*)c->B[c->cur].p;
          a.Din = (const float*)c->D[c->cur].p;
          a.Bout = (float*)c->B[1 - c->cur].p;
          a.Dout = (float*)c->D[1 - c->cur].p;
          if (plain_launch(c->prec, &a, (int)c->nz[i], c->cap_stream) != 0)
            cs = fail(c, GFDTD_E_CUDA, "plain launch failed");
        }
        if (!cs && plain_tick_launch((int*)c->d_plain_s.p, c->cap_stream) != 0)
          cs = fail(c, GFDTD_E_CUDA, "step counter launch failed");
        cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
        if (cs) { if (g) cudaGraphDestroy(g); return cs; }
        CK(c, e);
        cudaGraphExec_t ex = nullptr;
        e = cudaGraphInstantiate(&ex, g, 0);
        cudaGraphDestroy(g);
        CK(c, e);
        it = c->graphs.emplace(key, ex).first;
      }
      CK(c, cudaGraphLaunch(it->second, c->stream));
      c->launches += c->n_inst + 1;
      c->cur = 1 - c->cur;
    }
    s = enqueue_fold_advance(c, c->stream, ch, c->cur);
    if (s) return s;
    c->n_done += ch;
    n_steps -= ch;
  }
  return GFDTD_OK;
}

gfdtd_status gfdtd_plain_floor(gfdtd_ctx* c, int64_t n_steps) {
  if (!c) return GFDTD_E_ARG;
  if (c->prec == GFDTD_F32_KAHAN)
    return fail(c, GFDTD_E_UNSUPPORTED, "the plain kernel has no compensated tier");
  if (n_steps < 0) return fail(c, GFDTD_E_ARG, "n_steps < 0");
  gfdtd_status s = finalize(c);
  if (s) return s;
  if (c->n_tfsf > 0) return fail(c, GFDTD_E_UNSUPPORTED, "one-way sources run in gfdtd_step only");
  if (!c->d_plain_s.p) {
    s = dalloc(c, c->d_plain_s, 16);
    if (s) return s;
  }
  const auto key = std::make_pair(-2, c->cur);
  auto it = c->graphs.find(key);
  if (it == c->graphs.end()) {
    cudaGraph_t g = nullptr;
    CK(c, cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal));
    gfdtd_status cs = GFDTD_OK;
    for (int i = 0; i < c->n_inst && !cs; ++i) {
      char* Bp = (char*)c->B[c->cur].p + (size_t)c->off[i] * c->eb;
      char* Dp = (char*)c->D[c->cur].p + (size_t)c->off[i] * c->eb;
      if (plain_floor_launch(c->eb, Bp, Dp, (int)c->nz[i], (const int*)c->d_plain_s.p, c->cap_stream) != 0)
        cs = fail(c, GFDTD_E_CUDA, "floor launch failed");
    }
    if (!cs && plain_tick_launch((int*)c->d_plain_s.p, c->cap_stream) != 0)
      cs = fail(c, GFDTD_E_CUDA, "step counter launch failed");
    cudaError_t e = cudaStreamEndCapture(c->cap_stream, &g);
    if (cs) { if (g) cudaGraphDestroy(g); return cs; }
    CK(c, e);
    cudaGraphExec_t ex = nullptr;
    e = cudaGraphInstantiate(&ex, g, 0);
    cudaGraphDestroy(g);
    CK(c, e);
    it = c->graphs.emplace(key, ex).first;
  }
  CK(c, cudaMemsetAsync(c->d_plain_s.p, 0, sizeof(int), c->stream));
  for (int64_t st = 0; st < n_steps; ++st) {
    CK(c, cudaGraphLaunch(it->second, c->stream));
    c->launches += c->n_inst + 1;
  }
  return GFDTD_OK;
}

gfdtd_status gfdtd_read_fields(gfdtd_ctx* c, int inst, gfdtd_field which, double* dst, int64_t n) {
  gfdtd_status s = check_inst(c, inst);
  if (s) return s;
  if (!dst || n != c->nz[inst]) return fail(c, GFDTD_E_ARG, "n must equal nz and dst non-NULL");
  if (which < GFDTD_FIELD_D || which > GFDTD_FIELD_ESTAR) return fail(c, GFDTD_E_ARG, "bad field");
  if (which == GFDTD_FIELD_H && c->media[inst].kind == GFDTD_MATTER)
    return fail(c, GFDTD_E_UNSUPPORTED, "H is not available for moving matter");
  s = finalize(c);
  if (s) return s;
  s = dalloc(c, c->d_tmp, (size_t)n * sizeof(double));
  if (s) return s;
  const size_t o = (size_t)c->off[inst] * c->eb;
  if (which == GFDTD_FIELD_D || which == GFDTD_FIELD_B) {
    const DevBuf& b = which == GFDTD_FIELD_D ? c->D[c->cur] : c->B[c->cur];
    CKI(c, convert_launch(c->prec, 1, (const char*)b.p + o, c->d_tmp.p, n, c->stream));
  } else {
    CKI(c, derived_launch(c->prec, (int)which, (const InstDev*)c->d_inst.p, inst, tables_of(c),
                          c->B[c->cur].p, c->D[c->cur].p, (double*)c->d_tmp.p, (int)n, c->n_done,
                          c->stream));
  }
  CK(c, cudaMemcpyAsync(dst, c->d_tmp.p, (size_t)n * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return device_status(c);
}

gfdtd_status gfdtd_write_fields(gfdtd_ctx* c, int inst, gfdtd_field which, const double* src, int64_t n) {
  gfdtd_status s = check_inst(c, inst);
  if (s) return s;
  if (!src || n != c->nz[inst]) return fail(c, GFDTD_E_ARG, "n must equal nz and src non-NULL");
  if (which != GFDTD_FIELD_D && which != GFDTD_FIELD_B) return fail(c, GFDTD_E_ARG, "only D or B can be written");
  s = dalloc(c, c->d_tmp, (size_t)n * sizeof(double));
  if (s) return s;
  CK(c, cudaMemcpyAsync(c->d_tmp.p, src, (size_t)n * sizeof(double), cudaMemcpyHostToDevice, c->stream));
  const DevBuf& b = which == GFDTD_FIELD_D ? c->D[c->cur] : c->B[c->cur];
  CKI(c, convert_launch(c->prec, 0, c->d_tmp.p, (char*)b.p + (size_t)c->off[inst] * c->eb, n, c->stream));
  const DevBuf& cb = which == GFDTD_FIELD_D ? c->cD[c->cur] : c->cB[c->cur];
  if (cb.p) CK(c, cudaMemsetAsync((char*)cb.p + (size_t)c->off[inst] * c->eb, 0, (size_t)n * c->eb, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return GFDTD_OK;
}

gfdtd_status gfdtd_state_layout(const gfdtd_ctx* c, int64_t* n_elems, int* elem_bytes, int64_t* offsets) {
  if (!c) return GFDTD_E_ARG;
  if (n_elems) *n_elems = c->total;
  if (elem_bytes) *elem_bytes = c->eb;
  if (offsets) for (int i = 0; i < c->n_inst; ++i) offsets[i] = c->off[i];
  return GFDTD_OK;
}

gfdtd_status gfdtd_read_state(gfdtd_ctx* c, gfdtd_field which, void* dst, int64_t bytes) {
  if (!c) return GFDTD_E_ARG;
  if (which != GFDTD_FIELD_D && which != GFDTD_FIELD_B) return fail(c, GFDTD_E_ARG, "only D or B");
  if (!dst || bytes != c->total * c->eb) return fail(c, GFDTD_E_ARG, "bytes must be %lld", c->total * c->eb);
  const DevBuf& b = which == GFDTD_FIELD_D ? c->D[c->cur] : c->B[c->cur];
  CK(c, cudaMemcpyAsync(dst, b.p, (size_t)bytes, cudaMemcpyDeviceToHost, c->stream));
  return GFDTD_OK;
}

gfdtd_status gfdtd_write_state(gfdtd_ctx* c, gfdtd_field which, const void* src, int64_t bytes) {
  if (!c) return GFDTD_E_ARG;
  if (which != GFDTD_FIELD_D && which != GFDTD_FIELD_B) return fail(c, GFDTD_E_ARG, "only D or B");
  if (!src || bytes != c->total * c->eb) return fail(c, GFDTD_E_ARG, "bytes must be %lld", c->total * c->eb);
  const DevBuf& b = which == GFDTD_FIELD_D ? c->D[c->cur] : c->B[c->cur];
  CK(c, cudaMemcpyAsync(b.p, src, (size_t)bytes, cudaMemcpyHostToDevice, c->stream));
  const DevBuf& cb = which == GFDTD_FIELD_D ? c->cD[c->cur] : c->cB[c->cur];
  if (cb.p) CK(c, cudaMemsetAsync(cb.p, 0, (size_t)bytes, c->stream));
  return GFDTD_OK;
}

gfdtd_status gfdtd_read_spectrum(gfdtd_ctx* c, int inst, int probe_id, double* re, double* im) {
  gfdtd_status s = check_inst(c, inst);
  if (s) return s;
  if (probe_id < 0 || probe_id >= (int)c->inst_probes[inst].size() || !re || !im)
    return fail(c, GFDTD_E_ARG, "bad probe id or NULL output");
  s = finalize(c);
  if (s) return s;
  const int p = c->inst_probes[inst][probe_id];
  const int g = c->prb_global[p];
  const int b0 = c->prb_bin0[g];
  const size_t nb = c->probes[p].omega.size();
  CK(c, cudaMemcpyAsync(re, (double*)c->d_acc_re.p + b0, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaMemcpyAsync(im, (double*)c->d_acc_im.p + b0, nb * sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  return device_status(c);
}

gfdtd_status gfdtd_steps_done(const gfdtd_ctx* c, int64_t* n) {
  if (!c || !n) return GFDTD_E_ARG;
  *n = c->n_done;
  return GFDTD_OK;
}

gfdtd_status gfdtd_stability(double S, double beta, double eps_r, double mu_r, gfdtd_kind kind,
                             double* out) {
  if (!out || !(S > 0.0 && S <= 1.0) || !(beta > -1.0 && beta < 1.0) || !(eps_r > 0.0) || !(mu_r > 0.0))
    return GFDTD_E_ARG;
  if (kind != GFDTD_PERTURBATION && kind != GFDTD_MATTER) return GFDTD_E_ARG;
  double ie, im, bc;
  medium_coefs((int)kind, beta, eps_r, mu_r, &ie, &im, &bc);
  *out = max_zeta(S, beta, ie, im, bc);
  return GFDTD_OK;
}

gfdtd_status gfdtd_set_tuning(gfdtd_ctx* c, int cells_per_lane, int time_block, int blocks_per_sm) {
  if (!c) return GFDTD_E_ARG;
  if (cells_per_lane == 0 && time_block == 0) {
    c->C = 0;
    c->TB = 0;
    c->MB = 0;
    drop_graphs(c);
    return GFDTD_OK;
  }
  int Cs[16], TBs[16], MBs[16];
  const int n = block_shapes(c->prec, Cs, TBs, MBs, 16);
  for (int i = 0; i < n; ++i) {
    if (Cs[i] == cells_per_lane && TBs[i] == time_block &&
        (blocks_per_sm == 0 || MBs[i] == blocks_per_sm)) {
      gfdtd_status s = finalize(c);
      if (s) return s;
      c->split = true;
      return set_tiles(c, Cs[i], TBs[i], MBs[i]);
    }
  }
  return fail(c, GFDTD_E_UNSUPPORTED, "tile shape %d x %d (%d blocks/SM) not built for this precision",
              cells_per_lane, time_block, blocks_per_sm);
}

gfdtd_status gfdtd_get_stats(const gfdtd_ctx* c, gfdtd_stats* out) {
  if (!c || !out) return GFDTD_E_ARG;
  out->cells_per_lane = c->C;
  out->time_block = c->TB;
  out->blocks_per_sm = c->MB;
  out->n_tiles = (int64_t)c->n_tiles[0] + c->n_tiles[1] + c->n_tiles[2];
  out->kernel_launches = c->launches;
  long long cells = 0;
  for (long long v : c->nz) cells += v;
  out->cells = cells;
  out->uniform_split = c->split && c->prec != GFDTD_F32_KAHAN ? 1 : 0;
  return GFDTD_OK;
}

gfdtd_status gfdtd_watchdog(gfdtd_ctx* c, double limit, int reset, int* flags, double* amax) {
  if (!c) return GFDTD_E_ARG;
  if (!(limit > 0.0)) return fail(c, GFDTD_E_ARG, "limit must be > 0");
  std::vector<unsigned> w((size_t)c->n_inst);
  CK(c, cudaMemcpyAsync(w.data(), c->d_watch.p, w.size() * sizeof(unsigned), cudaMemcpyDeviceToHost,
                        c->stream));
  CK(c, cudaStreamSynchronize(c->stream));
  if (reset) CK(c, cudaMemsetAsync(c->d_watch.p, 0, w.size() * sizeof(unsigned), c->stream));
  int flagged = 0;
  for (int i = 0; i < c->n_inst; ++i) {
    // bits of an FP32 magnitude: above 0x7f800000 a NaN was written, at it an infinity
    const bool non_finite = w[i] >= 0x7f800000u;
    float m;
    const unsigned b = non_finite ? 0x7f800000u : w[i];
    std::memcpy(&m, &b, sizeof(float));
    const int f = (non_finite ? 1 : 0) | ((double)m > limit ? 2 : 0);
    if (flags) flags[i] = f;
    if (amax) amax[i] = (double)m;
    flagged += f != 0;
  }
  return flagged ? fail(c, GFDTD_E_UNSTABLE, "%d instance(s) flagged by the watchdog", flagged) : GFDTD_OK;
}

gfdtd_status gfdtd_test_stall(gfdtd_ctx* c, int on) {
  if (!c) return GFDTD_E_ARG;
  c->stall = on ? 1 : 0;
  drop_graphs(c);   // the flag is part of every captured launch
  return GFDTD_OK;
}

gfdtd_status gfdtd_synchronize(gfdtd_ctx* c) {
  if (!c) return GFDTD_E_ARG;
  CK(c, cudaStreamSynchronize(c->stream));
  return device_status(c);
}

const char* gfdtd_last_error(const gfdtd_ctx* c) {
  return c ? c->err.c_str() : g_create_error.c_str();
}

void gfdtd_destroy(gfdtd_ctx* c) {
  if (!c) return;
  cudaStreamSynchronize(c->stream);
  drop_graphs(c);
  DevBuf* bufs[] = {&c->B[0], &c->B[1], &c->D[0], &c->D[1], &c->cB[0], &c->cB[1], &c->cD[0],
                    &c->cD[1], &c->d_ndone, &c->d_inst, &c->d_zq,
                    &c->d_tabE, &c->d_tabH, &c->d_srcs, &c->d_prbs, &c->d_amp, &c->d_samples,
                    &c->d_omega, &c->d_binprb, &c->d_acc_re, &c->d_acc_im, &c->d_tiles[0],
                    &c->d_tiles[1], &c->d_tiles[2], &c->d_tmp, &c->d_tabE32, &c->d_tabH32, &c->d_ftiles, &c->d_track, &c->cap.buf,
                    &c->d_ckB, &c->d_ckD, &c->d_dseg[0], &c->d_dseg[1], &c->d_wB[0][0], &c->d_wB[0][1],
                    &c->d_wB[1][0], &c->d_wB[1][1], &c->d_amp2[0], &c->d_amp2[1], &c->d_lB[0],
                    &c->d_lB[1], &c->d_lD[0], &c->d_lD[1], &c->d_grad, &c->d_gn, &c->d_adjn[0], &c->d_adjn[1],
                    &c->d_Xre, &c->d_Xim, &c->d_bin0, &c->d_pnode, &c->d_acc0_re, &c->d_acc0_im,
                    &c->d_adj_tiles, &c->d_tfsf, &c->d_tfaux, &c->d_tfcorr, &c->d_watch, &c->d_watchblk, &c->d_plain_s, &c->d_queue};
  for (DevBuf* b : bufs) dfree(c, *b);
  if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
  delete c;
}

}  // extern "C"
