// vie_apply_noalloc: one operator apply that allocates no memory.
//
// Some callers cannot call cudaMalloc: a host application that gives each
// library a fixed device-memory budget and owns every allocation through its
// own pool, or a latency-critical loop where an allocation's implicit device
// synchronisation is not acceptable.  For them this entry point runs the same
// FP32 symmetric apply as vie_apply (S = 64 march, FP32 tiles, FP64 sums) on
// device buffers the caller owns, with every intermediate (padded sigma_t
// lattice, self-cell diagonal, source values, work list, work counter and the
// per-tile partial sums) in one file-scope device array of fixed size.
//
// The array is part of the library image: every GPU on which the library is
// loaded holds it until the process exits.  Its device address is looked up
// once per device (cudaGetSymbolAddress) on the first call made with that
// device current, and that first call also copies the self-cell quadrature
// rule to the device's constant memory (a synchronous copy), so the first
// call on each device should come before any stream capture.
// All calls on a device share its copy of the array, which keeps the last
// call's contents; the work counter is cleared on every call and nothing else
// needs to start at zero (every partial-sum slot is written before it is
// read).  Two calls whose work overlaps on the same GPU, for example on two
// streams, race on the array: serialise them.  The array takes about 17 MB:
// FP64 partial sums for 128 target tiles x 16384 cells plus small buffers.
#include <mutex>

#include "vie_internal.cuh"

namespace vie {

namespace {

constexpr long kNoallocMaxN = 16384;   // cells; 2D n <= 128, 3D n <= 25
constexpr int kTileCells = 128;        // target tile of the symmetric kernel
constexpr long kMaxT = (kNoallocMaxN + kTileCells - 1) / kTileCells;
constexpr long kMaxItems = kMaxT * (kMaxT + 1) / 2;
// Largest lattice for n^d <= 16384: 2D n = 128 pads to 129 x 129 (row stride
// 129), 3D n = 25 pads to 26^3; both fit in 26^3 = 17576 elements.
constexpr long kMaxLattice = 26L * 26 * 26;
constexpr long kMaxPadded = 26L * 26 * 26;

// byte offsets inside the scratch array (each 256-byte aligned)
constexpr size_t align256(size_t x) { return (x + 255) & ~size_t(255); }
constexpr size_t kOffPartial = 0;
constexpr size_t kOffDiag = align256(kOffPartial + sizeof(double) * kMaxT * kNoallocMaxN);
constexpr size_t kOffSrc = align256(kOffDiag + sizeof(double) * kNoallocMaxN);
constexpr size_t kOffPad32 = align256(kOffSrc + sizeof(float) * kNoallocMaxN);
constexpr size_t kOffPad64 = align256(kOffPad32 + sizeof(float) * kMaxPadded);
constexpr size_t kOffLattice = align256(kOffPad64 + sizeof(double) * kMaxPadded);
constexpr size_t kOffItems = align256(kOffLattice + sizeof(float) * kMaxLattice);
constexpr size_t kOffCounter = align256(kOffItems + sizeof(int2) * kMaxItems);
constexpr size_t kScratchBytes = align256(kOffCounter + 2 * sizeof(int));

static __device__ __align__(256) unsigned char g_scratch[kScratchBytes];

constexpr int kMaxDevices = 64;
std::mutex g_mu;
unsigned char *g_scratch_addr[kMaxDevices] = {};

// Work list of the symmetric kernel: item S(a) + (b - a) = (a, b), a <= b,
// S(a) = a T - a (a - 1) / 2.
__global__ void k_fill_items(int T, int2 *items) {
  const int a = blockIdx.x;
  const long base = (long)a * T - (long)a * (a - 1) / 2;
  for (int b = a + threadIdx.x; b < T; b += blockDim.x) items[base + (b - a)] = make_int2(a, b);
}

bool on_device(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

}  // namespace

}  // namespace vie

using namespace vie;

extern "C" vie_status vie_apply_noalloc(int dim, int n, const double *sigma_t, const double *sigma_s,
                                        vie_op op, const double *g, double *y, void *stream) {
  if (dim != 2 && dim != 3) {
    set_error("vie_apply_noalloc: dim must be 2 or 3");
    return VIE_ERR_INVALID_ARG;
  }
  const long N = dim == 2 ? (long)n * n : (long)n * n * n;
  if (n < 1 || N > kNoallocMaxN) {
    set_error("vie_apply_noalloc: n^dim must be in 1..16384 (the fixed scratch size)");
    return VIE_ERR_INVALID_ARG;
  }
  if (op != VIE_OP_K_SIGMA_S && op != VIE_OP_I_MINUS_K && op != VIE_OP_A_RAW) {
    set_error("vie_apply_noalloc: unknown op");
    return VIE_ERR_INVALID_ARG;
  }
  if (!sigma_t || !sigma_s || !g || !y || !on_device(sigma_t) || !on_device(sigma_s) ||
      !on_device(g) || !on_device(y)) {
    set_error("vie_apply_noalloc: sigma_t, sigma_s, g and y must be device pointers");
    return VIE_ERR_INVALID_ARG;
  }
  int dev = 0;
  VIE_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) {
    set_error("vie_apply_noalloc: device ordinal beyond the supported range");
    return VIE_ERR_INVALID_ARG;
  }
  unsigned char *base = nullptr;
  {
    std::lock_guard<std::mutex> lock(g_mu);
    if (!g_scratch_addr[dev]) {
      void *p = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&p, g_scratch);
      if (e != cudaSuccess) return cuda_fail(e, "vie_apply_noalloc: cudaGetSymbolAddress");
      g_scratch_addr[dev] = (unsigned char *)p;
    }
    base = g_scratch_addr[dev];
  }
  cudaStream_t st = (cudaStream_t)stream;
  double *partial = (double *)(base + kOffPartial);
  double *diag = (double *)(base + kOffDiag);
  float *src = (float *)(base + kOffSrc);
  float *pad32 = (float *)(base + kOffPad32);
  double *pad64 = (double *)(base + kOffPad64);
  float *lattice = (float *)(base + kOffLattice);
  int2 *items = (int2 *)(base + kOffItems);
  int *counter = (int *)(base + kOffCounter);

  vie_status s;
  if ((s = launch_pad_sigma(dim, n, sigma_t, pad32, pad64, st)) != VIE_OK) return s;
  SymPlan sp;
  if ((s = sym_plan_external(&sp, dim, n, N, pad32, dev, items, counter, lattice, kMaxLattice, (int)kMaxT, st)) !=
      VIE_OK)
    return s;
  if (!sp.usable) {
    set_error("vie_apply_noalloc: grid not supported by the shared-memory kernel");
    return VIE_ERR_UNSUPPORTED;
  }
  k_fill_items<<<sp.T, 128, 0, st>>>(sp.T, items);
  VIE_CHECK_LAUNCH("k_fill_items");
  VIE_CUDA(cudaMemsetAsync(counter, 0, 2 * sizeof(int), st));
  if ((s = launch_selfcell(dim, n, sigma_t, diag, st)) != VIE_OK) return s;
  if ((s = launch_source_prep(N, op, sigma_s, g, VIE_PREC_FP32, src, st)) != VIE_OK) return s;
  const double h = 1.0 / n;
  const float tau_scale2 = (float)(h / 64.0 * 1.4426950408889634);
  const float wcoef = (float)(dim == 2 ? h / (2.0 * kPi) : h / (4.0 * kPi));
  if ((s = sym_launch(sp, dim, n, N, tau_scale2, wcoef, src, partial, st)) != VIE_OK) return s;
  return launch_reduce(N, sp.T, op, partial, diag, sigma_s, g, y, st);
}
