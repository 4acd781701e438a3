// gfdtd_noalloc.cu -- gfdtd_step_noalloc: the batched time-block kernels run
// on caller-owned field buffers with every working buffer taken from one
// statically allocated device array, so the call allocates no memory.
//
// Who needs this: a caller whose device memory is not its own to allocate.
// A process whose GPU memory has been reserved up front by another framework's
// caching pool (a training or serving job) may find cudaMalloc failing, or
// may be forbidden to fragment that pool; a plugin host may hand its plugins
// buffers but no allocator; a loop with a fixed memory budget may not risk an
// allocation failing half way through a run.  For them this entry point
// advances one 1D instance with scratch that lives in a file-scope
// __device__ array sized for at most kMaxCells cells and kMaxValues profile
// values.  Every GPU that loads the library holds that array (about 4.4 MB)
// until the process exits.  The call synchronises its stream before it
// returns.
#include "../../include/gfdtd.h"
#include "gfdtd_block.cuh"
#include "gfdtd_medium.h"

#include <cmath>
#include <cstring>
#include <vector>

using namespace gfdtd;

namespace {

constexpr int kMaxCells = 1 << 18;                 // largest nz accepted
constexpr int kMaxValues = 1024;                   // largest number of profile values
constexpr int kC = 16, kTB = 16, kMB = 4;          // tile shape of the kernels used
constexpr int kMaxTiles = kMaxCells / tile_width(kC, kTB, true, 4) + 2;   // the narrower sign

// Byte layout of the scratch array (each region 256-byte aligned).
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kFieldBytes = align256(sizeof(float) * kMaxCells);
constexpr size_t kOffFields = 0;                                   // B0, D0, B1, D1
constexpr size_t kOffZq = kOffFields + 4 * kFieldBytes;
constexpr size_t kOffTabE = kOffZq + align256(sizeof(long long) * kMaxValues);
constexpr size_t kOffTabH = kOffTabE + align256(sizeof(double2) * kMaxValues);
constexpr size_t kOffTabE32 = kOffTabH + align256(sizeof(double2) * kMaxValues);
constexpr size_t kOffTabH32 = kOffTabE32 + align256(sizeof(float2) * kMaxValues);
constexpr size_t kOffTiles = kOffTabH32 + align256(sizeof(float2) * kMaxValues);
constexpr size_t kOffFast = kOffTiles + align256(3 * sizeof(int2) * kMaxTiles);
constexpr size_t kOffInst = kOffFast + align256(sizeof(FastTile) * kMaxTiles);
constexpr size_t kOffCounter = kOffInst + align256(sizeof(InstDev));
constexpr size_t kScratchBytes = kOffCounter + 256;

static __device__ __align__(256) unsigned char g_noalloc_scratch[kScratchBytes];

// Device address of g_noalloc_scratch per device, looked up on first use.
constexpr int kMaxDevices = 64;
void* g_scratch_addr[kMaxDevices] = {};

}  // namespace

extern "C" gfdtd_status gfdtd_step_noalloc(int64_t nz, double S, gfdtd_kind kind, double beta,
                                           gfdtd_interp interp, int n, const double* z,
                                           const double* eps_r, const double* mu_r, float* B,
                                           float* D, int64_t n_done, int64_t n_steps,
                                           void* cuda_stream) {
  // ---- arguments (the same rules as gfdtd_create + gfdtd_set_medium)
  if (nz < 1 || nz > kMaxCells) return GFDTD_E_ARG;          // beyond the scratch array
  if (n < 1 || n > kMaxValues || (interp == GFDTD_LINEAR && n < 2)) return GFDTD_E_ARG;
  if (!(S > 0.0 && S <= 1.0) || !(beta > -1.0 && beta < 1.0) || std::fabs(beta) * S >= 1.0)
    return GFDTD_E_ARG;
  if (kind != GFDTD_PERTURBATION && kind != GFDTD_MATTER) return GFDTD_E_ARG;
  if (interp != GFDTD_LAYERS && interp != GFDTD_LINEAR) return GFDTD_E_ARG;
  if (!eps_r || !mu_r || !B || !D || n_done < 0 || n_steps < 0) return GFDTD_E_ARG;
  const int npos = interp == GFDTD_LAYERS ? n - 1 : n;
  if (npos > 0 && !z) return GFDTD_E_ARG;
  for (int i = 0; i < n; ++i)
    if (!(eps_r[i] > 0.0) || !(mu_r[i] > 0.0)) return GFDTD_E_ARG;
  for (int i = 1; i < npos; ++i)
    if (!(z[i] > z[i - 1])) return GFDTD_E_ARG;
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // ---- scratch address on this device (looked up by the first call on each device)
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= kMaxDevices) return GFDTD_E_CUDA;
  if (!g_scratch_addr[dev]) {
    void* p = nullptr;
    if (cudaGetSymbolAddress(&p, g_noalloc_scratch) != cudaSuccess || !p) return GFDTD_E_CUDA;
    g_scratch_addr[dev] = p;
  }
  unsigned char* base = static_cast<unsigned char*>(g_scratch_addr[dev]);
  float* fld[4];
  for (int k = 0; k < 4; ++k) fld[k] = reinterpret_cast<float*>(base + kOffFields + k * kFieldBytes);

  // ---- the instance and its tables, built on the host exactly as the context path builds them
  InstDev I{};
  I.off = 0;
  I.nz = (int)nz;
  I.nz_pad = (int)((nz + 31) / 32 * 32);
  MediumSpec ms;
  ms.kind = (int)kind;
  ms.beta = beta;
  ms.interp = (int)interp;
  ms.n = n;
  ms.z = z;
  ms.eps = eps_r;
  ms.mu = mu_r;
  std::vector<long long> zq;
  std::vector<double2> tE, tH;
  std::vector<float2> tE32, tH32;
  fill_instance(ms, S, I, zq, tE, tH, tE32, tH32);
  const int flags = I.flags;
  // tiles by kernel variant, as the context path lists them
  std::vector<int2> tiles[3];
  std::vector<FastTile> fast;          // records of tiles[2] (this call has no sources or probes)
  {
    const bool pos = (flags & F_POS) != 0;
    const int W = tile_width(kC, kTB, pos, 4);
    const int L = tile_margin(kTB, pos, 4);
    for (long long x0 = 0; x0 < nz; x0 += W) {
      const long long b0 = x0 - L;
      const bool edge = b0 < 0 || b0 + 32LL * kC > nz;
      const int v = (flags & F_MATTER) ? 1 : (fast_eligible(I, kC) && !edge ? 2 : 0);
      tiles[v].push_back(make_int2(0, (int)x0));
      if (v == 2) {
        FastTile f{};
        f.e = b0;
        f.inst = 0;
        f.x0 = (int)x0;
        f.base = (int)b0;
        fast.push_back(f);
      }
    }
  }

  // ---- upload; clear the field buffers so cells past nz start (and stay) zero
  const size_t fbytes = sizeof(float) * (size_t)I.nz_pad;
#define NA_CK(x) do { if ((x) != cudaSuccess) return GFDTD_E_CUDA; } while (0)
  for (int k = 0; k < 4; ++k) NA_CK(cudaMemsetAsync(fld[k], 0, fbytes, st));
  NA_CK(cudaMemcpyAsync(fld[0], B, sizeof(float) * nz, cudaMemcpyDeviceToDevice, st));
  NA_CK(cudaMemcpyAsync(fld[1], D, sizeof(float) * nz, cudaMemcpyDeviceToDevice, st));
  NA_CK(cudaMemcpyAsync(base + kOffZq, zq.data(), sizeof(long long) * n, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(base + kOffTabE, tE.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(base + kOffTabH, tH.data(), sizeof(double2) * n, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(base + kOffTabE32, tE32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(base + kOffTabH32, tH32.data(), sizeof(float2) * n, cudaMemcpyHostToDevice, st));
  for (int v = 0; v < 3; ++v)
    if (!tiles[v].empty())
      NA_CK(cudaMemcpyAsync(base + kOffTiles + v * sizeof(int2) * kMaxTiles, tiles[v].data(),
                            sizeof(int2) * tiles[v].size(), cudaMemcpyHostToDevice, st));
  if (!fast.empty())
    NA_CK(cudaMemcpyAsync(base + kOffFast, fast.data(), sizeof(FastTile) * fast.size(),
                          cudaMemcpyHostToDevice, st));
  NA_CK(cudaMemcpyAsync(base + kOffInst, &I, sizeof(InstDev), cudaMemcpyHostToDevice, st));
  long long counter[2] = {n_done, 0};                 // steps done; status word
  NA_CK(cudaMemcpyAsync(base + kOffCounter, counter, sizeof(counter), cudaMemcpyHostToDevice, st));

  // ---- time blocks, ping-ponging between the two halves of the scratch fields
  int num_sms = 0;
  NA_CK(cudaDeviceGetAttribute(&num_sms, cudaDevAttrMultiProcessorCount, dev));
  int cur = 0;
  for (long long s0 = 0; s0 < n_steps; s0 += kTB) {
    for (int v = 0; v < 3; ++v) {
      if (tiles[v].empty()) continue;
      BlockArgs<float> a{};
      a.inst = reinterpret_cast<const InstDev*>(base + kOffInst);
      a.tiles = reinterpret_cast<const int2*>(base + kOffTiles + v * sizeof(int2) * kMaxTiles);
      a.n_tiles = (int)tiles[v].size();
      a.tb.zq = reinterpret_cast<const long long*>(base + kOffZq);
      a.tb.tabE = reinterpret_cast<const double2*>(base + kOffTabE);
      a.tb.tabH = reinterpret_cast<const double2*>(base + kOffTabH);
      a.tb.tabE32 = reinterpret_cast<const float2*>(base + kOffTabE32);
      a.tb.tabH32 = reinterpret_cast<const float2*>(base + kOffTabH32);
      a.Bin = fld[2 * cur];
      a.Din = fld[2 * cur + 1];
      a.Bout = fld[2 * (1 - cur)];
      a.Dout = fld[2 * (1 - cur) + 1];
      a.n_done = reinterpret_cast<const long long*>(base + kOffCounter);
      a.err = reinterpret_cast<int*>(base + kOffCounter + 8);
      a.s0 = (int)s0;
      a.nsteps = (int)std::min<long long>(kTB, n_steps - s0);
      a.record = 0;
      if (v == 2) a.ftiles = reinterpret_cast<const FastTile*>(base + kOffFast);
      const int grid = std::max(1, std::min(num_sms * kMB, (a.n_tiles + 3) / 4));
      if (block_launch(GFDTD_F32, v, kC, kTB, kMB, &a, grid, 128, st) != 0) return GFDTD_E_CUDA;
    }
    cur = 1 - cur;
  }
  // status first: on a failed bounded wait the caller's B and D are left as they were
  NA_CK(cudaMemcpyAsync(counter, base + kOffCounter, sizeof(counter), cudaMemcpyDeviceToHost, st));
  NA_CK(cudaStreamSynchronize(st));
  if ((int)counter[1] & 0xff) return GFDTD_E_TIMEOUT;
  NA_CK(cudaMemcpyAsync(B, fld[2 * cur], sizeof(float) * nz, cudaMemcpyDeviceToDevice, st));
  NA_CK(cudaMemcpyAsync(D, fld[2 * cur + 1], sizeof(float) * nz, cudaMemcpyDeviceToDevice, st));
  NA_CK(cudaStreamSynchronize(st));
#undef NA_CK
  return GFDTD_OK;
}
