// C ABI of the VIE library: handle management, operator apply, the FP64
// GMRES driver (Algorithm 1, S.2) and the step-two sweep (Algorithm 1, S.3).
// Everything numeric runs in the kernels of k_apply.cu, k_krylov.cu and
// k_sweep.cu; this file validates arguments, owns device memory, stages host
// buffers and sequences launches on the caller's stream.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <string>
#include <vector>

#include "vie_internal.cuh"

namespace vie {

static thread_local std::string g_last_error;
// vie_set_wait_limits: milliseconds (first < 0: the same as limit)
static std::atomic<double> g_wait_ms{1000.0}, g_first_wait_ms{-1.0};

vie_status get_dev_props(int device, DevProps *out) {
  static std::atomic<int> sms_cache[64], optin_cache[64];
  int sms = device >= 0 && device < 64 ? sms_cache[device].load() : 0;
  int optin = device >= 0 && device < 64 ? optin_cache[device].load() : 0;
  if (sms <= 0 || optin <= 0) {
    VIE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, device));
    VIE_CUDA(cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, device));
    if (device >= 0 && device < 64) {
      sms_cache[device].store(sms);
      optin_cache[device].store(optin);
    }
  }
  out->sharedMemPerBlockOptin = (size_t)optin;
  out->multiProcessorCount = sms;
  return VIE_OK;
}

WaitLimits wait_limits(int device) {
  // the clock-rate query is slow (a driver round trip): once per device
  static std::atomic<int> khz_cache[64];
  int khz = device >= 0 && device < 64 ? khz_cache[device].load() : 0;
  if (khz <= 0) {
    if (cudaDeviceGetAttribute(&khz, cudaDevAttrClockRate, device) != cudaSuccess || khz <= 0) khz = 2000000;
    if (device >= 0 && device < 64) khz_cache[device].store(khz);
  }
  const double ms = g_wait_ms.load(), fms = g_first_wait_ms.load();
  WaitLimits w;
  w.limit = (long long)(ms * khz);
  w.first = fms < 0.0 ? w.limit : (long long)(fms * khz);
  return w;
}
static std::atomic<unsigned long long> g_launches{0};

void count_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }

void set_error(const std::string &msg) { g_last_error = msg; }

vie_status cuda_fail(cudaError_t e, const char *what) {
  set_error(std::string(what) + ": " + cudaGetErrorName(e) + " (" + cudaGetErrorString(e) + ")");
  return e == cudaErrorMemoryAllocation ? VIE_ERR_OOM : VIE_ERR_CUDA;
}

static vie_status invalid(const std::string &msg) {
  set_error(msg);
  return VIE_ERR_INVALID_ARG;
}

// Select the handle's device for the duration of a call, then restore the
// caller's current device.
struct DeviceGuard {
  int prev = -1;
  cudaError_t err = cudaSuccess;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    err = cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

static bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  cudaError_t e = cudaPointerGetAttributes(&at, p);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

template <typename T>
static vie_status dalloc(T **p, size_t count) {
  *p = nullptr;
  if (count == 0) return VIE_OK;
  cudaError_t e = vie_malloc((void **)p, count * sizeof(T));
  if (e != cudaSuccess) {
    *p = nullptr;
    return cuda_fail(e, "cudaMalloc");
  }
  return VIE_OK;
}

template <typename T>
static void dfree(T *&p) {
  if (p) vie_free((void *)p);
  p = nullptr;
}

// A growable device buffer.
template <typename T>
struct DBuf {
  T *ptr = nullptr;
  size_t count = 0;
  vie_status reserve(size_t want) {
    if (want <= count) return VIE_OK;
    dfree(ptr);
    count = 0;
    vie_status s = dalloc(&ptr, want);
    if (s == VIE_OK) count = want;
    return s;
  }
  void release() {
    dfree(ptr);
    count = 0;
  }
};

// Events around one operator apply: [0] start, [1] before the pair kernel,
// [2] after it, [3] end.
struct ApplyEvents {
  cudaEvent_t e[4] = {nullptr, nullptr, nullptr, nullptr};
  bool pending = false;
};

// Workspace of R GMRES(m) solves in lockstep (vie_gmres_opts.nrhs > 1):
// the KBatch arrays plus the bases V [R][m + 1][N], the flexible directions
// Z [R][m][N], phi, r, w [R][N], the steps per solve kk [R], pinned host
// copies of the scalars and of gv, and the network input [R][3][N].
struct MultiGmres {
  int R = 0, m = 0, has_z = 0, has_net = 0;
  KBatch kb{};
  double *V = nullptr, *Z = nullptr, *phi = nullptr, *r = nullptr, *w = nullptr;
  int *kk = nullptr;
  double *h_scal = nullptr, *h_gv = nullptr;
  int *h_act = nullptr;
  float *net_x = nullptr;
};

}  // namespace vie

using namespace vie;

struct vie_handle {
  int device = 0;
  int dim = 2, n = 1, P = 2;
  long N = 1;
  vie_opts opts{};
  double *sig_t = nullptr, *sig_s = nullptr;  // FP64 [N]
  float *sig32 = nullptr;                     // padded FP32 lattice
  double *sig64 = nullptr;                    // padded FP64 lattice
  double *diag = nullptr;                     // self-cell d_j [N]
  Medium med{};
  PairPlan plan{};
  SymPlan sym{};                              // symmetric kernel, when usable
  DispPlan disp{};                            // displacement-major kernel, when usable
  DispPlan3 disp3{};                          // its 3D form, when usable
  FftPre fft{};                               // FFT preconditioner (Section 4.4), when set
  DiffPre diff{};                             // diffusion preconditioner (Section 4.4), when set
  FmmPlan fmm{};                              // FMM operator (Section 3.3), when assembled
  int use_kernel = VIE_KERNEL_GENERAL;        // pair kernel chosen for applies
  void *src = nullptr;                        // per-source values [N]
  double *partial = nullptr;                  // [plan.splits][N]
  DBuf<double> stage_a, stage_b, stage_c;     // host-pointer staging
  DBuf<float> stage_f1, stage_f2;
  float *qpad = nullptr;                      // sweep source lattice
  // GMRES workspace
  int gm_m = 0;
  double *V = nullptr, *phi = nullptr, *r = nullptr, *w = nullptr, *H = nullptr;
  double *cs = nullptr, *sn = nullptr, *gv = nullptr, *yv = nullptr, *hcol = nullptr;
  double *htmp = nullptr, *part = nullptr, *scal = nullptr;
  double *h_pinned = nullptr;                 // host-pinned scalars / gv seed
  // apply timing
  bool opts_disable_sym = false;              // force the general kernel (tests)
  // assembled operator
  int asm_mode = VIE_OPERATOR_OTF;
  void *pairs = nullptr;                      // pair weights the dense assembly expands (displacement kernel)
  float *sym_partial = nullptr;               // row/column sums of the symmetric blocks (VIE_OPERATOR_SYM32)
  long ldk = 0;
  void *kmat = nullptr;                       // FP32 K or BF16 Khi
  void *kmat_lo = nullptr;                    // BF16 Klo
  DBuf<float> g32;                            // FP32 copy of a right-hand side
  DBuf<unsigned char> gemm_ws;                // split-K partials + BF16 G
  int *dev_err = nullptr;                     // device error word of the products
  int *ticket = nullptr;                      // block ticket of the fused dot kernels (0 between launches)
  bool sig_s_positive = false;                // phi = K (f / sigma_s) is available
  UnetImpl *precond = nullptr;                // learned right preconditioner
  double precond_inv_ref = 0.2;
  bool precond_on_diff = false;               // the network corrects the diffusion preconditioner's z
  double *Z = nullptr;                        // FGMRES: preconditioned basis [m][N]
  int z_m = 0;
  float *net_x = nullptr;                     // network input [3][N]
  DBuf<double> fscaled;                       // f / sigma_s
  std::vector<ApplyEvents> events;
  size_t ev_next = 0;
  double t_apply_ms = 0.0, t_kernel_ms = 0.0;
  int n_apply = 0;
  MultiGmres mg;                              // lockstep solves of several right-hand sides
  int *h_err = nullptr;                       // pinned copies of the device error words [2]
};

namespace {

void free_gmres(vie_handle *h) {
  dfree(h->V);
  dfree(h->phi);
  dfree(h->r);
  dfree(h->w);
  dfree(h->H);
  dfree(h->cs);
  dfree(h->sn);
  dfree(h->gv);
  dfree(h->yv);
  dfree(h->hcol);
  dfree(h->htmp);
  dfree(h->part);
  dfree(h->scal);
  if (h->h_pinned) vie_free_host(h->h_pinned);
  h->h_pinned = nullptr;
  h->gm_m = 0;
}

void free_multi(MultiGmres &g) {
  KBatch &b = g.kb;
  for (double **p : {&g.V, &g.Z, &g.phi, &g.r, &g.w, &b.H, &b.cs, &b.sn, &b.gv, &b.yv, &b.hcol, &b.htmp, &b.part,
                     &b.scal, &b.bnorm})
    dfree(*p);
  for (int **p : {&b.ticket, &b.act, &g.kk}) dfree(*p);
  dfree(g.net_x);
  if (g.h_scal) vie_free_host(g.h_scal);
  if (g.h_gv) vie_free_host(g.h_gv);
  if (g.h_act) vie_free_host(g.h_act);
  g = MultiGmres{};
}

void free_all(vie_handle *h) {
  dfree(h->sig_t);
  dfree(h->sig_s);
  dfree(h->sig32);
  dfree(h->sig64);
  dfree(h->diag);
  if (h->src) vie_free(h->src);
  h->src = nullptr;
  if (h->pairs) vie_free(h->pairs);
  h->pairs = nullptr;
  if (h->sym_partial) vie_free(h->sym_partial);
  h->sym_partial = nullptr;
  dfree(h->partial);
  h->stage_a.release();
  h->stage_b.release();
  h->stage_c.release();
  h->stage_f1.release();
  h->stage_f2.release();
  dfree(h->qpad);
  dfree(h->Z);
  dfree(h->net_x);
  if (h->kmat) vie_free(h->kmat);
  if (h->kmat_lo) vie_free(h->kmat_lo);
  h->kmat = h->kmat_lo = nullptr;
  h->g32.release();
  h->gemm_ws.release();
  dfree(h->dev_err);
  dfree(h->ticket);
  sym_release(&h->sym);
  disp_release(&h->disp);
  fft_release(&h->fft);
  diffusion_release(&h->diff);
  fmm_release(&h->fmm);
  disp3_release(&h->disp3);
  free_gmres(h);
  free_multi(h->mg);
  if (h->h_err) vie_free_host(h->h_err);
  h->h_err = nullptr;
  for (auto &ev : h->events)
    for (auto &e : ev.e)
      if (e) cudaEventDestroy(e);
  h->events.clear();
}

vie_status ensure_gmres(vie_handle *h, int m) {
  if (h->gm_m >= m) return VIE_OK;
  free_gmres(h);
  const long N = h->N;
  const int blocks = dot_blocks(N);
  vie_status s;
  if ((s = dalloc(&h->V, (size_t)(m + 1) * N)) != VIE_OK) return s;
  if ((s = dalloc(&h->phi, N)) != VIE_OK) return s;
  if ((s = dalloc(&h->r, N)) != VIE_OK) return s;
  if ((s = dalloc(&h->w, N)) != VIE_OK) return s;
  if ((s = dalloc(&h->H, (size_t)(m + 1) * m)) != VIE_OK) return s;
  if ((s = dalloc(&h->cs, m)) != VIE_OK) return s;
  if ((s = dalloc(&h->sn, m)) != VIE_OK) return s;
  if ((s = dalloc(&h->gv, m + 1)) != VIE_OK) return s;
  if ((s = dalloc(&h->yv, m)) != VIE_OK) return s;
  if ((s = dalloc(&h->hcol, m + 1)) != VIE_OK) return s;
  if ((s = dalloc(&h->htmp, m + 1)) != VIE_OK) return s;
  if ((s = dalloc(&h->part, (size_t)blocks * (m + 1))) != VIE_OK) return s;
  if ((s = dalloc(&h->scal, 8)) != VIE_OK) return s;
  if (!h->ticket) {
    if ((s = dalloc(&h->ticket, 1)) != VIE_OK) return s;
    VIE_CUDA(cudaMemset(h->ticket, 0, sizeof(int)));
  }
  VIE_CUDA(vie_malloc_host((void **)&h->h_pinned, sizeof(double) * (m + 1 + 8)));
  h->gm_m = m;
  return VIE_OK;
}

vie_status harvest_events(vie_handle *h) {
  for (auto &ev : h->events) {
    if (!ev.pending) continue;
    VIE_CUDA(cudaEventSynchronize(ev.e[3]));
    float a = 0.f, k = 0.f;
    VIE_CUDA(cudaEventElapsedTime(&a, ev.e[0], ev.e[3]));
    VIE_CUDA(cudaEventElapsedTime(&k, ev.e[1], ev.e[2]));
    h->t_apply_ms += a;
    h->t_kernel_ms += k;
    ev.pending = false;
  }
  return VIE_OK;
}

// One operator application on device vectors.
vie_status apply_dev(vie_handle *h, int op, const double *g, double *y, cudaStream_t st,
                     bool timed) {
  ApplyEvents *ev = nullptr;
  if (timed) {
    if (h->events.empty()) {
      h->events.resize(8);
      for (auto &e : h->events)
        for (auto &x : e.e) VIE_CUDA(cudaEventCreate(&x));
    }
    ev = &h->events[h->ev_next];
    if (ev->pending) {
      vie_status s = harvest_events(h);
      if (s != VIE_OK) return s;
    }
    h->ev_next = (h->ev_next + 1) % h->events.size();
    VIE_CUDA(cudaEventRecord(ev->e[0], st));
  }
  const int prec = h->opts.precision;
  const int closed = h->opts.tau_mode == VIE_TAU_CLOSED;
  const bool raw_via_k = op == VIE_OP_A_RAW && h->sig_s_positive;
  if (h->asm_mode == VIE_OPERATOR_FMM) {
    vie_status s = launch_source_prep(h->N, op, h->sig_s, g, VIE_PREC_FP32, h->src, st);
    if (s != VIE_OK) return s;
    if (timed) VIE_CUDA(cudaEventRecord(ev->e[1], st));
    if ((s = fmm_apply(h->fmm, op, (const float *)h->src, g, y, st)) != VIE_OK) return s;
    if (timed) {
      VIE_CUDA(cudaEventRecord(ev->e[2], st));
      VIE_CUDA(cudaEventRecord(ev->e[3], st));
      ev->pending = true;
    }
    h->n_apply++;
    return VIE_OK;
  }
  if (h->asm_mode == VIE_OPERATOR_SYM32) {
    if (timed) VIE_CUDA(cudaEventRecord(ev->e[1], st));
    vie_status s = h->dim == 3 ? symv3_apply(h->disp3, op, h->sig_s, g, (const float *)h->kmat, (float *)h->src,
                                             h->sym_partial, y, h->device, st)
                               : symv_apply(h->n, op, h->sig_s, g, (const float *)h->kmat, (float *)h->src,
                                            h->sym_partial, y, h->device, st);
    if (s != VIE_OK) return s;
    if (timed) {
      VIE_CUDA(cudaEventRecord(ev->e[2], st));
      VIE_CUDA(cudaEventRecord(ev->e[3], st));
      ev->pending = true;
    }
    h->n_apply++;
    return VIE_OK;
  }
  const bool dense = h->asm_mode == VIE_OPERATOR_FP32 || h->asm_mode == VIE_OPERATOR_BF16X3;
  if (dense && (op != VIE_OP_A_RAW || raw_via_k)) {
    vie_status s = h->g32.reserve(h->ldk);
    if (s != VIE_OK) return s;
    if (raw_via_k) {
      // phi = A f = K (sigma_s^{-1} f)  (Eq. EQ:ERT Intgrl FMM)
      if ((s = h->fscaled.reserve(h->N)) != VIE_OK) return s;
      if ((s = launch_divide(h->N, g, h->sig_s, h->fscaled.ptr, st)) != VIE_OK) return s;
      g = h->fscaled.ptr;
      op = VIE_OP_K_SIGMA_S;
    }
    if (timed) VIE_CUDA(cudaEventRecord(ev->e[1], st));
    s = launch_gemv(h->kmat, h->kmat_lo, h->asm_mode == VIE_OPERATOR_BF16X3, h->ldk, h->N, g,
                    h->g32.ptr, op, y, st);
    if (s != VIE_OK) return s;
    if (timed) {
      VIE_CUDA(cudaEventRecord(ev->e[2], st));
      VIE_CUDA(cudaEventRecord(ev->e[3], st));
      ev->pending = true;
    }
    h->n_apply++;
    return VIE_OK;
  }
  if (h->use_kernel == VIE_KERNEL_DISPLACEMENT && h->dim == 3) {
    const double hh = 1.0 / h->n;
    vie_status s = disp3_apply(h->disp3, op, h->sig_s, g, h->diag, (float *)h->src,
                               (float)(hh / h->opts.steps * 1.4426950408889634), (float)(hh / (4.0 * kPi)), y,
                               timed ? ev->e[1] : nullptr, timed ? ev->e[2] : nullptr, st);
    if (s != VIE_OK) return s;
    if (timed) {
      VIE_CUDA(cudaEventRecord(ev->e[3], st));
      ev->pending = true;
    }
    h->n_apply++;
    return VIE_OK;
  }
  vie_status s = h->use_kernel == VIE_KERNEL_DISPLACEMENT
                     ? disp_source(h->disp, h->N, op, h->sig_s, g, (float *)h->src, st)
                     : launch_source_prep(h->N, op, h->sig_s, g, prec, h->src, st);
  if (s != VIE_OK) return s;
  if (timed) VIE_CUDA(cudaEventRecord(ev->e[1], st));
  int slots = h->plan.splits;
  const double hh = 1.0 / h->n;
  const float tau_scale2 = (float)(hh / h->opts.steps * 1.4426950408889634);
  const float wcoef = (float)(h->dim == 2 ? hh / (2.0 * kPi) : hh / (4.0 * kPi));
  if (h->use_kernel == VIE_KERNEL_DISPLACEMENT) {
    if (h->asm_mode == VIE_OPERATOR_PAIRS32) {
      s = disp_stream(h->disp, h->n, (const float *)h->kmat, (const float *)h->src, st);
    } else {
      s = disp_launch(h->disp, h->n, tau_scale2, wcoef, (const float *)h->src, st);
    }
  } else if (h->use_kernel == VIE_KERNEL_SYMMETRIC) {
    s = sym_launch(h->sym, h->dim, h->n, h->N, tau_scale2, wcoef, (const float *)h->src,
                   h->partial, st);
    slots = h->sym.T;
  } else {
    s = launch_pairs(h->med, h->plan, h->opts.steps, closed, prec, h->src, h->partial, st);
  }
  if (s != VIE_OK) return s;
  if (timed) VIE_CUDA(cudaEventRecord(ev->e[2], st));
  s = h->use_kernel == VIE_KERNEL_DISPLACEMENT
          ? disp_reduce(h->disp, h->N, op, h->diag, h->sig_s, g, y, st)
          : launch_reduce(h->N, slots, op, h->partial, h->diag, h->sig_s, g, y, st);
  if (s != VIE_OK) return s;
  if (timed) {
    VIE_CUDA(cudaEventRecord(ev->e[3], st));
    ev->pending = true;
  }
  h->n_apply++;
  return VIE_OK;
}

// ||x||^2 into dev scalar *out (part: dot partials buffer).
vie_status norm2_dev(vie_handle *h, const double *x, double *out, cudaStream_t st) {
  const int blocks = dot_blocks(h->N);
  vie_status s = launch_dots(x, 1, h->N, x, h->N, h->part, blocks, st);
  if (s != VIE_OK) return s;
  return launch_dots_finish(h->part, blocks, 1, out, 0, st);
}

// Device error words of the handle's tensor-core kernels (the product's and
// the learned preconditioner's): queue their copies to pinned memory before a
// synchronisation, then take_errors reports VIE_ERR_TIMEOUT if a bounded
// device wait gave up (and clears the words for the next call).
vie_status queue_errors(vie_handle *h, cudaStream_t st) {
  if (!h->h_err) VIE_CUDA(vie_malloc_host((void **)&h->h_err, 2 * sizeof(int)));
  h->h_err[0] = h->h_err[1] = 0;
  if (h->dev_err) VIE_CUDA(cudaMemcpyAsync(h->h_err, h->dev_err, sizeof(int), cudaMemcpyDeviceToHost, st));
  if (h->precond)
    VIE_CUDA(cudaMemcpyAsync(h->h_err + 1, unet_error_word(h->precond), sizeof(int), cudaMemcpyDeviceToHost, st));
  return VIE_OK;
}

vie_status take_errors(vie_handle *h, cudaStream_t st) {
  if (!h->h_err || (h->h_err[0] == 0 && h->h_err[1] == 0)) return VIE_OK;
  if (h->h_err[0] && h->dev_err) VIE_CUDA(cudaMemsetAsync(h->dev_err, 0, sizeof(int), st));
  if (h->h_err[1] && h->precond) VIE_CUDA(cudaMemsetAsync(unet_error_word(h->precond), 0, sizeof(int), st));
  VIE_CUDA(cudaStreamSynchronize(st));
  h->h_err[0] = h->h_err[1] = 0;
  set_error("a tensor-core kernel gave up on a bounded device wait (its output is NaN)");
  return VIE_ERR_TIMEOUT;
}

vie_status read_scalar(vie_handle *h, const double *dev, double *val, cudaStream_t st) {
  VIE_CUDA(cudaMemcpyAsync(h->h_pinned, dev, sizeof(double), cudaMemcpyDeviceToHost, st));
  vie_status s = queue_errors(h, st);
  if (s != VIE_OK) return s;
  VIE_CUDA(cudaStreamSynchronize(st));
  *val = h->h_pinned[0];
  return take_errors(h, st);
}

bool all_finite(const double *a, long n) {
  for (long i = 0; i < n; ++i)
    if (!isfinite(a[i])) return false;
  return true;
}

vie_status ensure_multi(vie_handle *h, int R, int m, bool need_z, bool need_net) {
  MultiGmres &g = h->mg;
  if (g.R >= R && g.m >= m && (g.has_z || !need_z) && (g.has_net || !need_net)) return VIE_OK;
  free_multi(g);
  const long N = h->N;
  const int blocks = dot_blocks(N);
  KBatch &b = g.kb;
  vie_status s;
  if ((s = dalloc(&g.V, (size_t)R * (m + 1) * N)) != VIE_OK) return s;
  if (need_z && (s = dalloc(&g.Z, (size_t)R * m * N)) != VIE_OK) return s;
  if ((s = dalloc(&g.phi, (size_t)R * N)) != VIE_OK) return s;
  if ((s = dalloc(&g.r, (size_t)R * N)) != VIE_OK) return s;
  if ((s = dalloc(&g.w, (size_t)R * N)) != VIE_OK) return s;
  if ((s = dalloc(&b.H, (size_t)R * (m + 1) * m)) != VIE_OK) return s;
  if ((s = dalloc(&b.cs, (size_t)R * m)) != VIE_OK) return s;
  if ((s = dalloc(&b.sn, (size_t)R * m)) != VIE_OK) return s;
  if ((s = dalloc(&b.gv, (size_t)R * (m + 1))) != VIE_OK) return s;
  if ((s = dalloc(&b.yv, (size_t)R * m)) != VIE_OK) return s;
  if ((s = dalloc(&b.hcol, (size_t)R * (m + 1))) != VIE_OK) return s;
  if ((s = dalloc(&b.htmp, (size_t)R * (m + 1))) != VIE_OK) return s;
  if ((s = dalloc(&b.part, (size_t)R * blocks * (m + 1))) != VIE_OK) return s;
  if ((s = dalloc(&b.scal, (size_t)R * 8)) != VIE_OK) return s;
  if ((s = dalloc(&b.bnorm, (size_t)R)) != VIE_OK) return s;
  if ((s = dalloc(&b.ticket, (size_t)R)) != VIE_OK) return s;
  if ((s = dalloc(&b.act, (size_t)R)) != VIE_OK) return s;
  if ((s = dalloc(&g.kk, (size_t)R)) != VIE_OK) return s;
  if (need_net && (s = dalloc(&g.net_x, (size_t)R * 3 * N)) != VIE_OK) return s;
  VIE_CUDA(cudaMemset(b.ticket, 0, sizeof(int) * R));
  VIE_CUDA(vie_malloc_host((void **)&g.h_scal, sizeof(double) * 8 * R));
  VIE_CUDA(vie_malloc_host((void **)&g.h_gv, sizeof(double) * (size_t)R * (m + 1)));
  VIE_CUDA(vie_malloc_host((void **)&g.h_act, sizeof(int) * 2 * R));
  g.R = R;
  g.m = m;
  g.has_z = need_z;
  g.has_net = need_net;
  b.N = N;
  b.m = m;
  b.R = R;
  b.blocks = blocks;
  return VIE_OK;
}

// Operator applies to R vectors, column r of g at g + r ldg and of y at
// y + r ldy.  With the assembled BF16 hi/lo operator every product of K goes
// through the tensor cores, all columns in one product (up to 128); otherwise
// one apply per column with act[r] != 0 (act NULL: every column).
vie_status apply_multi(vie_handle *h, int op, const double *g, long ldg, double *y, long ldy, int R,
                       const int *act, cudaStream_t st, bool timed) {
  vie_status s;
  if (h->asm_mode == VIE_OPERATOR_BF16X3 && op != VIE_OP_A_RAW) {
    ApplyEvents *ev = nullptr;
    if (timed) {
      if (h->events.empty()) {
        h->events.resize(8);
        for (auto &e : h->events)
          for (auto &x : e.e) VIE_CUDA(cudaEventCreate(&x));
      }
      ev = &h->events[h->ev_next];
      if (ev->pending && (s = harvest_events(h)) != VIE_OK) return s;
      h->ev_next = (h->ev_next + 1) % h->events.size();
      VIE_CUDA(cudaEventRecord(ev->e[0], st));
      VIE_CUDA(cudaEventRecord(ev->e[1], st));
    }
    int sms = 0;
    VIE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    for (int r0 = 0; r0 < R; r0 += kGemmMaxRhs) {
      const int nr = std::min(kGemmMaxRhs, R - r0);
      if ((s = h->gemm_ws.reserve(gemm_workspace_bytes(h->N, h->ldk, nr, nullptr, sms))) != VIE_OK) return s;
      if ((s = launch_gemm_bf16x3(h->kmat, h->kmat_lo, h->ldk, h->N, g + (size_t)r0 * ldg, ldg, nr, op,
                                  y + (size_t)r0 * ldy, ldy, h->gemm_ws.ptr, h->dev_err, st)) != VIE_OK)
        return s;
    }
    if (timed) {
      VIE_CUDA(cudaEventRecord(ev->e[2], st));
      VIE_CUDA(cudaEventRecord(ev->e[3], st));
      ev->pending = true;
    }
    h->n_apply++;
    return VIE_OK;
  }
  for (int r = 0; r < R; ++r)
    if (!act || act[r])
      if ((s = apply_dev(h, op, g + (size_t)r * ldg, y + (size_t)r * ldy, st, timed)) != VIE_OK) return s;
  return VIE_OK;
}

// act[] to the device (from pageable memory: the call returns once the host
// values are staged, so the vector may change right after)
vie_status upload_act(vie_handle *h, const std::vector<int> &act, cudaStream_t st) {
  VIE_CUDA(cudaMemcpyAsync(h->mg.kb.act, act.data(), sizeof(int) * act.size(), cudaMemcpyHostToDevice, st));
  return VIE_OK;
}

// scal[8 r + slot] of every r, after the work queued so far
vie_status read_multi_scal(vie_handle *h, int R, cudaStream_t st) {
  MultiGmres &g = h->mg;
  VIE_CUDA(cudaMemcpyAsync(g.h_scal, g.kb.scal, sizeof(double) * 8 * R, cudaMemcpyDeviceToHost, st));
  vie_status s = queue_errors(h, st);
  if (s != VIE_OK) return s;
  VIE_CUDA(cudaStreamSynchronize(st));
  return take_errors(h, st);
}

// R restarted GMRES(m) / FGMRES solves of (I - K) U_r = phi_r in lockstep
// (Algorithm 1, S.2 for several sources on one medium): every Arnoldi step
// applies the operator to the R current directions at once (one tensor-core
// product with the assembled BF16 hi/lo operator), runs CGS2, the norms and
// the Givens steps of all R in one launch each, and reads the R residual
// estimates back in one copy.  A solve leaves the step loop when its estimate
// reaches rtol (or it stalls under a preconditioner, or maxit), the others go
// on; restart cycles, the true FP64 residual and convergence are per solve,
// exactly as in the single solve.
vie_status solve_multi(vie_handle *h, const double *fdev, double *x, int R, const vie_gmres_opts &opt,
                       vie_report *rep, cudaStream_t st, bool timed,
                       std::chrono::steady_clock::time_point t_start) {
  const long N = h->N;
  const int m = opt.restart;
  const bool has_precond = h->precond || h->fft.on || h->diff.on;
  vie_status s;
  if ((s = ensure_multi(h, R, m, has_precond, h->precond != nullptr)) != VIE_OK) return s;
  MultiGmres &g = h->mg;
  KBatch b = g.kb;
  b.R = R;
  b.m = m;
  const long ldv = (long)(m + 1) * N, ldz = (long)m * N;
  std::vector<int> act(R, 1), conv(R, 0), iters(R, 0), restarts(R, 0), napply(R, 0), pit(R, 0), fell(R, 0);
  std::vector<int> done(R, 0);  // maxit reached and the final true residual taken
  std::vector<int> kk(R, 0);
  std::vector<double> bnorm(R, 0.0), relres(R, 0.0), est(R, 0.0);
  if ((s = upload_act(h, act, st)) != VIE_OK) return s;
  // phi_r = A f_r (Eq. EQ:ERT Intgrl FMM), unless the caller passed phi
  if (opt.rhs_is_phi) {
    VIE_CUDA(cudaMemcpyAsync(g.phi, fdev, sizeof(double) * R * N, cudaMemcpyDeviceToDevice, st));
  } else if (h->asm_mode == VIE_OPERATOR_BF16X3 && h->sig_s_positive) {
    // phi_r = K (f_r / sigma_s) for every r in one tensor-core product
    if ((s = launch_divide_cols(N, R, fdev, N, h->sig_s, g.w, N, st)) != VIE_OK) return s;
    if ((s = apply_multi(h, VIE_OP_K_SIGMA_S, g.w, N, g.phi, N, R, nullptr, st, timed)) != VIE_OK) return s;
    for (int r = 0; r < R; ++r) ++napply[r];
  } else {
    for (int r = 0; r < R; ++r)
      if ((s = apply_dev(h, VIE_OP_A_RAW, fdev + (size_t)r * N, g.phi + (size_t)r * N, st, timed)) != VIE_OK)
        return s;
    for (int r = 0; r < R; ++r) ++napply[r];
  }
  if ((s = launch_bnorm2(b, g.phi, N, 0, st)) != VIE_OK) return s;
  if ((s = read_multi_scal(h, R, st)) != VIE_OK) return s;
  for (int r = 0; r < R; ++r) {
    const double bn2 = g.h_scal[8 * r];
    if (!isfinite(bn2)) {
      set_error("vie_solve_gmres: non-finite right-hand side");
      return VIE_ERR_NONFINITE;
    }
    bnorm[r] = sqrt(bn2);
    if (bnorm[r] == 0.0) {
      VIE_CUDA(cudaMemsetAsync(x + (size_t)r * N, 0, sizeof(double) * N, st));
      conv[r] = 1;
    }
  }
  VIE_CUDA(cudaMemcpyAsync(b.bnorm, bnorm.data(), sizeof(double) * R, cudaMemcpyHostToDevice, st));
  bool x_is_zero = opt.zero_x0 != 0;
  for (;;) {
    for (int r = 0; r < R; ++r) act[r] = !conv[r] && !done[r];
    if (std::none_of(act.begin(), act.end(), [](int a) { return a != 0; })) break;
    if ((s = upload_act(h, act, st)) != VIE_OK) return s;
    // true residuals r = phi - (I - K) x
    if (x_is_zero) {
      VIE_CUDA(cudaMemcpyAsync(g.r, g.phi, sizeof(double) * R * N, cudaMemcpyDeviceToDevice, st));
    } else {
      if ((s = apply_multi(h, VIE_OP_I_MINUS_K, x, N, g.w, N, R, act.data(), st, timed)) != VIE_OK) return s;
      for (int r = 0; r < R; ++r) napply[r] += act[r];
      if ((s = launch_baxpby(b, 1.0, g.phi, N, -1.0, g.w, N, g.r, N, st)) != VIE_OK) return s;
    }
    x_is_zero = false;
    if ((s = launch_bnorm2(b, g.r, N, 1, st)) != VIE_OK) return s;
    if ((s = read_multi_scal(h, R, st)) != VIE_OK) return s;
    for (int r = 0; r < R; ++r) {
      if (!act[r]) continue;
      const double rn2 = g.h_scal[8 * r + 1];
      if (!isfinite(rn2)) {
        set_error("vie_solve_gmres: non-finite residual");
        return VIE_ERR_NONFINITE;
      }
      relres[r] = sqrt(rn2) / bnorm[r];
      if (relres[r] <= opt.rtol) conv[r] = 1;
      if (!conv[r] && iters[r] >= opt.maxit) done[r] = 1;
      if (conv[r] || done[r]) act[r] = 0;
    }
    if (std::none_of(act.begin(), act.end(), [](int a) { return a != 0; })) break;
    if ((s = upload_act(h, act, st)) != VIE_OK) return s;
    // V_r0 = r_r / beta_r, gv_r = beta_r e_1
    if ((s = launch_bscale(b, g.r, N, 1, 1, g.V, ldv, st)) != VIE_OK) return s;
    for (int r = 0; r < R; ++r) {
      double *gv = g.h_gv + (size_t)r * (m + 1);
      for (int i = 0; i <= m; ++i) gv[i] = 0.0;
      gv[0] = act[r] ? sqrt(g.h_scal[8 * r + 1]) : 0.0;
    }
    VIE_CUDA(cudaMemcpyAsync(b.gv, g.h_gv, sizeof(double) * R * (m + 1), cudaMemcpyHostToDevice, st));
    const std::vector<int> cycle = act;  // the solves that take part in this cycle
    std::fill(kk.begin(), kk.end(), 0);
    std::vector<double> est_prev(R, 1e300), est_prev2(R, 1e300);
    std::vector<int> stall(R, 0);
    const bool flexible = has_precond;
    for (int k = 0; k < m; ++k) {
      if (std::none_of(act.begin(), act.end(), [](int a) { return a != 0; })) break;
      const double *op_in = g.V + (size_t)k * N;
      long ld_in = ldv;
      if (flexible) {
        // z_r,k = M(v_r,k) (right preconditioning, flexible GMRES); a solve
        // whose preconditioned iteration stalled goes on with M = I
        double *zk = g.Z + (size_t)k * N;
        if (h->precond) {
          if (h->precond_on_diff)  // the diffusion preconditioner first; the network corrects it
            for (int r = 0; r < R; ++r)
              if (act[r] && !fell[r] &&
                  (s = diffusion_precondition(h->diff, g.V + (size_t)r * ldv + (size_t)k * N, zk + (size_t)r * ldz,
                                              st)) != VIE_OK)
                return s;
          if ((s = launch_bnorm2(b, g.V + (size_t)k * N, ldv, 4, st)) != VIE_OK) return s;
          if ((s = unet_precondition_batch(h->precond, h->sig_t, h->sig_s, h->precond_inv_ref, g.V + (size_t)k * N,
                                           ldv, b.scal, 4, R, h->n, g.net_x, h->precond_on_diff ? zk : nullptr,
                                           ldz, zk, ldz, st)) != VIE_OK)
            return s;
        } else {
          for (int r = 0; r < R; ++r) {
            if (!act[r] || fell[r]) continue;
            const double *vr = g.V + (size_t)r * ldv + (size_t)k * N;
            double *zr = zk + (size_t)r * ldz;
            if (h->fft.on)
              s = fft_precondition(h->fft, vr, zr, st);
            else
              s = diffusion_precondition(h->diff, vr, zr, st);
            if (s != VIE_OK) return s;
          }
        }
        for (int r = 0; r < R; ++r) {
          if (act[r] && fell[r])
            VIE_CUDA(cudaMemcpyAsync(zk + (size_t)r * ldz, g.V + (size_t)r * ldv + (size_t)k * N,
                                     sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
          if (act[r] && !fell[r]) ++pit[r];
        }
        op_in = zk;
        ld_in = ldz;
      }
      double *vk1 = g.V + (size_t)(k + 1) * N;
      if ((s = apply_multi(h, VIE_OP_I_MINUS_K, op_in, ld_in, vk1, ldv, R, act.data(), st, timed)) != VIE_OK)
        return s;
      for (int r = 0; r < R; ++r) napply[r] += act[r];
      // CGS2 (two passes of h = V^T w, w -= V h), the norm and the Givens step
      if ((s = launch_bdots(b, g.V, ldv, k + 1, vk1, ldv, b.hcol, nullptr, st)) != VIE_OK) return s;
      if ((s = launch_borth_update(b, g.V, ldv, k + 1, b.hcol, vk1, ldv, st)) != VIE_OK) return s;
      if ((s = launch_bdots(b, g.V, ldv, k + 1, vk1, ldv, b.htmp, b.hcol, st)) != VIE_OK) return s;
      if ((s = launch_borth_update(b, g.V, ldv, k + 1, b.htmp, vk1, ldv, st)) != VIE_OK) return s;
      if ((s = launch_bnorm2_givens(b, vk1, ldv, k, st)) != VIE_OK) return s;
      if ((s = launch_bscale(b, vk1, ldv, 2, 1, vk1, ldv, st)) != VIE_OK) return s;
      if ((s = read_multi_scal(h, R, st)) != VIE_OK) return s;
      if (timed && (s = harvest_events(h)) != VIE_OK) return s;
      bool changed = false;
      for (int r = 0; r < R; ++r) {
        if (!act[r]) continue;
        const double e = g.h_scal[8 * r + 3];
        ++iters[r];
        kk[r] = k + 1;
        est[r] = e;
        if (!isfinite(e)) {
          if (!flexible || fell[r]) {
            set_error("vie_solve_gmres: non-finite Arnoldi step");
            return VIE_ERR_NONFINITE;
          }
          --kk[r];  // the preconditioner produced a non-finite direction: drop this step
          stall[r] = 1;
        } else if (flexible && !fell[r] && k >= 1 && e > 0.8 * est_prev[r] && est_prev[r] > 0.8 * est_prev2[r]) {
          stall[r] = 1;
        }
        if (stall[r] || e <= opt.rtol || iters[r] >= opt.maxit) {
          act[r] = 0;
          changed = true;
        }
        est_prev2[r] = est_prev[r];
        est_prev[r] = e;
      }
      if (changed && (s = upload_act(h, act, st)) != VIE_OK) return s;
    }
    // x_r += V_r y_r (or Z_r y_r) for every solve of the cycle with steps
    std::vector<int> upd(R, 0);
    for (int r = 0; r < R; ++r) upd[r] = cycle[r] && kk[r] > 0;
    if ((s = upload_act(h, upd, st)) != VIE_OK) return s;
    VIE_CUDA(cudaMemcpyAsync(g.kk, kk.data(), sizeof(int) * R, cudaMemcpyHostToDevice, st));
    if ((s = launch_bupdate(b, flexible ? g.Z : g.V, flexible ? ldz : ldv, g.kk, x, N, st)) != VIE_OK) return s;
    // the cycle's host vectors must outlive the copies above
    VIE_CUDA(cudaStreamSynchronize(st));
    for (int r = 0; r < R; ++r) {
      if (!cycle[r]) continue;
      ++restarts[r];
      if (stall[r]) fell[r] = 1;
    }
  }
  VIE_CUDA(cudaStreamSynchronize(st));
  if (timed && (s = harvest_events(h)) != VIE_OK) return s;
  const double t_total =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  bool all_conv = true;
  for (int r = 0; r < R; ++r) {
    all_conv = all_conv && conv[r];
    if (!rep) continue;
    vie_report &Q = rep[r];
    Q = vie_report{};
    Q.iters = iters[r];
    Q.restarts = restarts[r];
    Q.converged = conv[r];
    Q.n_apply = napply[r];
    Q.relres = relres[r];
    Q.relres_est = est[r];
    Q.t_total_ms = t_total;
    Q.t_apply_ms = h->t_apply_ms;
    Q.t_apply_kernel_ms = h->t_kernel_ms;
    Q.precond_iters = pit[r];
    Q.fell_back = fell[r];
  }
  if (!all_conv) {
    set_error("vie_solve_gmres: maxit reached before rtol for some right-hand sides");
    return VIE_ERR_NOT_CONVERGED;
  }
  return VIE_OK;
}

}  // namespace

extern "C" {

const char *vie_last_error(void) { return g_last_error.c_str(); }

const char *vie_version(void) { return "vie-gb300 0.2 (sm_103a; M-iii/M-ii, FMM, FFT/diffusion/learned preconditioners)"; }

unsigned long long vie_kernel_launches(void) { return g_launches.load(); }

void vie_default_opts(vie_opts *o) {
  if (!o) return;
  o->steps = 64;
  o->tau_mode = VIE_TAU_MARCH;
  o->precision = VIE_PREC_FP32;
  o->device = 0;
  o->kernel = VIE_KERNEL_AUTO;
  o->disc = VIE_DISC_MIII;
}

void vie_default_gmres_opts(vie_gmres_opts *o) {
  if (!o) return;
  o->rtol = 1e-6;
  o->restart = 64;
  o->maxit = 1000;
  o->zero_x0 = 1;
  o->rhs_is_phi = 0;
  o->time_apply = 0;
  o->nrhs = 1;
}

vie_status vie_create(vie_handle **out, const vie_grid *g, const double *sigma_t,
                      const double *sigma_s, const vie_opts *o) {
  g_last_error.clear();
  if (!out || !g || !sigma_t || !sigma_s) return invalid("vie_create: NULL argument");
  *out = nullptr;
  vie_opts opts;
  vie_default_opts(&opts);
  if (o) opts = *o;
  if (g->dim != 2 && g->dim != 3) return invalid("vie_create: dim must be 2 or 3");
  if (g->n < 1 || (g->dim == 2 && g->n > 4096) || (g->dim == 3 && g->n > 256))
    return invalid("vie_create: n out of range (2D: 1..4096, 3D: 1..256)");
  if (opts.steps < 1 || opts.steps > 4096) return invalid("vie_create: steps must be in 1..4096");
  if (opts.tau_mode != VIE_TAU_MARCH && opts.tau_mode != VIE_TAU_CLOSED)
    return invalid("vie_create: unknown tau_mode");
  if (opts.precision != VIE_PREC_FP32 && opts.precision != VIE_PREC_FP64)
    return invalid("vie_create: unknown precision");
  if (opts.kernel < VIE_KERNEL_AUTO || opts.kernel > VIE_KERNEL_GENERAL)
    return invalid("vie_create: unknown kernel");
  if (opts.disc != VIE_DISC_MIII && opts.disc != VIE_DISC_MII) return invalid("vie_create: unknown disc");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || ndev == 0) {
    cudaGetLastError();
    set_error("vie_create: no CUDA device");
    return VIE_ERR_CUDA;
  }
  if (opts.device < 0 || opts.device >= ndev) return invalid("vie_create: bad device ordinal");
  const long N = g->dim == 2 ? (long)g->n * g->n : (long)g->n * g->n * g->n;
  if (is_device_ptr(sigma_t) || is_device_ptr(sigma_s))
    return invalid("vie_create: sigma_t and sigma_s must be host arrays");
  bool ss_positive = true;
  for (long i = 0; i < N; ++i) {
    ss_positive = ss_positive && sigma_s[i] > 0.0;
    if (!isfinite(sigma_t[i]) || !isfinite(sigma_s[i])) {
      set_error("vie_create: non-finite coefficient");
      return VIE_ERR_NONFINITE;
    }
    if (sigma_t[i] < 0.0 || sigma_s[i] < 0.0) return invalid("vie_create: negative coefficient");
    if (opts.tau_mode == VIE_TAU_CLOSED && sigma_t[i] != sigma_t[0])
      return invalid("vie_create: VIE_TAU_CLOSED needs a constant sigma_t");
  }
  DeviceGuard dg(opts.device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  vie_handle *h = new vie_handle();
  h->device = opts.device;
  h->dim = g->dim;
  h->n = g->n;
  h->P = g->n + 1;
  h->N = N;
  h->opts = opts;
  h->sig_s_positive = ss_positive;
  const long lattice = g->dim == 2 ? (long)h->P * h->P : (long)h->P * h->P * h->P;
  vie_status s;
#define TRY(x)            \
  do {                    \
    s = (x);              \
    if (s != VIE_OK) {    \
      free_all(h);        \
      delete h;           \
      return s;           \
    }                     \
  } while (0)
  TRY(dalloc(&h->sig_t, N));
  TRY(dalloc(&h->sig_s, N));
  TRY(dalloc(&h->sig32, lattice));
  TRY(dalloc(&h->sig64, lattice));
  TRY(dalloc(&h->diag, N));
  cudaStream_t st = 0;
  auto cpy = [&](void *d, const void *src, size_t bytes) -> vie_status {
    VIE_CUDA(cudaMemcpy(d, src, bytes, cudaMemcpyHostToDevice));
    return VIE_OK;
  };
  TRY(cpy(h->sig_t, sigma_t, sizeof(double) * N));
  TRY(cpy(h->sig_s, sigma_s, sizeof(double) * N));
  TRY(launch_pad_sigma(g->dim, g->n, h->sig_t, h->sig32, h->sig64, st));
  TRY(launch_selfcell(g->dim, g->n, h->sig_t, h->diag, st));
  h->med.dim = g->dim;
  h->med.n = g->n;
  h->med.P = h->P;
  h->med.N = N;
  h->med.sig32 = h->sig32;
  h->med.sig64 = h->sig64;
  h->med.sigma_c = sigma_t[0];
  TRY(plan_pairs(h->med, opts.steps, opts.tau_mode == VIE_TAU_CLOSED, opts.precision,
                 opts.device, &h->plan));
  {
    size_t bytes = (opts.precision == VIE_PREC_FP64 ? sizeof(double) : sizeof(float)) * N;
    cudaError_t e = vie_malloc(&h->src, bytes);
    if (e != cudaSuccess) TRY(cuda_fail(e, "cudaMalloc"));
  }
  const bool fast = opts.precision == VIE_PREC_FP32 && opts.tau_mode == VIE_TAU_MARCH && opts.steps == 64;
  if (fast && opts.kernel != VIE_KERNEL_GENERAL) {
    TRY(sym_prepare(&h->sym, g->dim, g->n, N, h->sig32, opts.device, st));
    if (g->dim == 2 && (opts.kernel == VIE_KERNEL_AUTO || opts.kernel == VIE_KERNEL_DISPLACEMENT))
      TRY(disp_prepare(&h->disp, g->n, h->sig32, opts.device, st));
    if (g->dim == 3 && (opts.kernel == VIE_KERNEL_AUTO || opts.kernel == VIE_KERNEL_DISPLACEMENT))
      TRY(disp3_prepare(&h->disp3, g->n, h->sig32, opts.device, st));
  }
  if ((h->disp.usable || h->disp3.usable) && opts.kernel != VIE_KERNEL_SYMMETRIC)
    h->use_kernel = VIE_KERNEL_DISPLACEMENT;
  else if (h->sym.usable)
    h->use_kernel = VIE_KERNEL_SYMMETRIC;
  else
    h->use_kernel = VIE_KERNEL_GENERAL;
  if (opts.disc == VIE_DISC_MII) {
    // M-ii: the displacement kernel with per-D weights, and the diagonal
    // (h / 2 pi) times the cell integral at t = 0 for every cell
    if (g->dim != 2 || h->use_kernel != VIE_KERNEL_DISPLACEMENT) {
      free_all(h);
      delete h;
      set_error("vie_create: VIE_DISC_MII needs a 2D grid with FP32 tiles, the S = 64 march and the "
                "displacement kernel (n <= 258)");
      return VIE_ERR_UNSUPPORTED;
    }
    double dval = 0.0;
    TRY(disp_mii_prepare(&h->disp, g->n, &dval, st));
    std::vector<double> dv((size_t)N, dval);
    TRY(cpy(h->diag, dv.data(), sizeof(double) * N));
  }
  {
    long slots = h->plan.splits;
    if (h->use_kernel == VIE_KERNEL_SYMMETRIC) slots = std::max<long>(slots, h->sym.T);
    TRY(dalloc(&h->partial, (size_t)slots * N));
  }
  {
    cudaError_t e = cudaDeviceSynchronize();
    if (e != cudaSuccess) TRY(cuda_fail(e, "vie_create setup kernels"));
  }
#undef TRY
  *out = h;
  return VIE_OK;
}

vie_status vie_destroy(vie_handle *h) {
  if (!h) return VIE_OK;
  DeviceGuard dg(h->device);
  cudaDeviceSynchronize();
  {
    DeviceIdle idle;  // synchronised just above: the buffers go back to the cache at once
    free_all(h);
  }
  delete h;
  return VIE_OK;
}

vie_status vie_get_kernel(vie_handle *h, int *kernel) {
  if (!h || !kernel) return invalid("vie_get_kernel: NULL argument");
  *kernel = h->opts.precision == VIE_PREC_FP32 ? h->use_kernel : VIE_KERNEL_GENERAL;
  return VIE_OK;
}

vie_status vie_get_kernel_work(vie_handle *h, double *fma_per_apply) {
  if (!h || !fma_per_apply) return invalid("vie_get_kernel_work: NULL argument");
  int k = VIE_KERNEL_GENERAL;
  vie_get_kernel(h, &k);
  const double pairs = 0.5 * (double)h->N * (double)(h->N - 1);
  *fma_per_apply = k != VIE_KERNEL_DISPLACEMENT ? pairs * h->opts.steps * (h->dim == 3 ? 7.0 : 3.0)
                   : h->dim == 3                ? h->disp3.taps
                                                : h->disp.taps;
  return VIE_OK;
}

vie_status vie_get_diagonal(vie_handle *h, double *d, void *stream) {
  if (!h || !d) return invalid("vie_get_diagonal: NULL argument");
  DeviceGuard dg(h->device);
  cudaStream_t st = (cudaStream_t)stream;
  if (is_device_ptr(d)) {
    VIE_CUDA(cudaMemcpyAsync(d, h->diag, sizeof(double) * h->N, cudaMemcpyDeviceToDevice, st));
  } else {
    VIE_CUDA(cudaMemcpyAsync(d, h->diag, sizeof(double) * h->N, cudaMemcpyDeviceToHost, st));
    VIE_CUDA(cudaStreamSynchronize(st));
  }
  return VIE_OK;
}

vie_status vie_apply(vie_handle *h, vie_op op, const double *g, double *y, int nrhs,
                     void *stream) {
  if (!h || !g || !y) return invalid("vie_apply: NULL argument");
  if (op != VIE_OP_K_SIGMA_S && op != VIE_OP_I_MINUS_K && op != VIE_OP_A_RAW)
    return invalid("vie_apply: unknown op");
  if (nrhs < 1) return invalid("vie_apply: nrhs must be >= 1");
  DeviceGuard dg(h->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const long N = h->N;
  const size_t total = (size_t)nrhs * N;
  const bool gd = is_device_ptr(g), yd = is_device_ptr(y);
  const double *gg = g;
  double *yy = y;
  vie_status s;
  if (!gd) {
    if ((s = h->stage_a.reserve(total)) != VIE_OK) return s;
    VIE_CUDA(cudaMemcpyAsync(h->stage_a.ptr, g, sizeof(double) * total, cudaMemcpyHostToDevice, st));
    gg = h->stage_a.ptr;
  }
  if (!yd) {
    if ((s = h->stage_b.reserve(total)) != VIE_OK) return s;
    yy = h->stage_b.ptr;
  }
  if (h->asm_mode == VIE_OPERATOR_BF16X3 && op != VIE_OP_A_RAW && nrhs >= 2) {
    int sms = 0;
    VIE_CUDA(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, h->device));
    for (int r0 = 0; r0 < nrhs; r0 += kGemmMaxRhs) {
      const int nr = std::min(kGemmMaxRhs, nrhs - r0);
      if ((s = h->gemm_ws.reserve(gemm_workspace_bytes(N, h->ldk, nr, nullptr, sms))) != VIE_OK)
        return s;
      if ((s = launch_gemm_bf16x3(h->kmat, h->kmat_lo, h->ldk, N, gg + (size_t)r0 * N, N, nr, op,
                                  yy + (size_t)r0 * N, N, h->gemm_ws.ptr, h->dev_err, st)) != VIE_OK)
        return s;
      h->n_apply += nr;
    }
  } else {
    for (int r = 0; r < nrhs; ++r)
      if ((s = apply_dev(h, op, gg + (size_t)r * N, yy + (size_t)r * N, st, false)) != VIE_OK)
        return s;
  }
  if (!yd) {
    VIE_CUDA(cudaMemcpyAsync(y, yy, sizeof(double) * total, cudaMemcpyDeviceToHost, st));
    if ((s = queue_errors(h, st)) != VIE_OK) return s;
    VIE_CUDA(cudaStreamSynchronize(st));
    return take_errors(h, st);
  }
  return VIE_OK;
}

vie_status vie_check_device(vie_handle *h, void *stream) {
  if (!h) return invalid("vie_check_device: NULL handle");
  DeviceGuard dg(h->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  vie_status s = queue_errors(h, st);
  if (s != VIE_OK) return s;
  VIE_CUDA(cudaStreamSynchronize(st));
  return take_errors(h, st);
}

vie_status vie_set_wait_limits(double limit_ms, double first_wait_ms) {
  if (!(limit_ms > 0.0) || limit_ms > 60000.0 || !(first_wait_ms <= limit_ms))
    return invalid("vie_set_wait_limits: 0 < limit_ms <= 60000 and first_wait_ms <= limit_ms required");
  g_wait_ms = limit_ms;
  g_first_wait_ms = first_wait_ms < 0.0 ? -1.0 : first_wait_ms;
  return VIE_OK;
}

static vie_status assemble_impl(vie_handle *h, int mode, int order, void *stream) {
  if (!h) return invalid("vie_assemble: NULL handle");
  if (mode != VIE_OPERATOR_OTF && mode != VIE_OPERATOR_FP32 && mode != VIE_OPERATOR_BF16X3 &&
      mode != VIE_OPERATOR_PAIRS32 && mode != VIE_OPERATOR_SYM32 && mode != VIE_OPERATOR_FMM)
    return invalid("vie_assemble: unknown mode");
  DeviceGuard dg(h->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const bool reuse = mode != VIE_OPERATOR_OTF && mode != VIE_OPERATOR_FMM && mode == h->asm_mode && h->kmat;
  if (!reuse) {
    if (h->kmat || h->kmat_lo || h->fmm.on) VIE_CUDA(cudaStreamSynchronize(st));
    if (h->kmat) vie_free(h->kmat);
    if (h->kmat_lo) vie_free(h->kmat_lo);
    h->kmat = h->kmat_lo = nullptr;
    fmm_release(&h->fmm);
    h->asm_mode = VIE_OPERATOR_OTF;
  }
  if (mode == VIE_OPERATOR_OTF) return VIE_OK;
  if (mode == VIE_OPERATOR_FMM) {
    // the interpolation-based FMM of Section 3.3 with cached kernel values
    if (h->dim != 2 || h->opts.precision != VIE_PREC_FP32 || h->opts.disc != VIE_DISC_MIII) {
      set_error("vie_assemble: VIE_OPERATOR_FMM needs a 2D grid, FP32 tiles and M-iii");
      return VIE_ERR_UNSUPPORTED;
    }
    vie_status s = fmm_prepare(&h->fmm, h->n, order, h->sig32, h->diag, h->opts.steps,
                               h->opts.tau_mode == VIE_TAU_CLOSED, h->med.sigma_c, st);
    if (s != VIE_OK) {
      fmm_release(&h->fmm);
      return s;
    }
    h->asm_mode = mode;
    return VIE_OK;
  }
  if (mode == VIE_OPERATOR_SYM32 && h->dim == 3) {
    // A in the symmetric blocks of grid-line pairs: the 3D pair weights, expanded
    if (h->use_kernel != VIE_KERNEL_DISPLACEMENT || !h->disp3.usable || h->opts.disc != VIE_DISC_MIII) {
      set_error("vie_assemble: VIE_OPERATOR_SYM32 in 3D needs the 3D displacement kernel (FP32 tiles, S = 64, "
                "n <= 32)");
      return VIE_ERR_UNSUPPORTED;
    }
    long bf = 0, pf = 0;
    vie_status s = disp3_sym_sizes(&h->disp3, h->device, &bf, &pf);
    if (s != VIE_OK) return s;
    if (!reuse) VIE_CUDA(vie_malloc(&h->kmat, sizeof(float) * (size_t)bf));
    if (!h->sym_partial) VIE_CUDA(vie_malloc((void **)&h->sym_partial, sizeof(float) * (size_t)pf));
    const double hh = 1.0 / h->n;
    s = disp3_assemble(&h->disp3, (float)(hh / h->opts.steps * 1.4426950408889634), (float)(hh / (4.0 * kPi)),
                       h->sig_s, h->diag, 0, (float *)h->kmat, nullptr, nullptr, h->device, st);
    if (s != VIE_OK) return s;
    h->asm_mode = mode;
    return VIE_OK;
  }
  if (mode == VIE_OPERATOR_SYM32) {
    // A in the symmetric blocks of grid-row pairs: the pair weights, expanded
    if (h->use_kernel != VIE_KERNEL_DISPLACEMENT || h->dim != 2 || !disp_expand_fits(h->n, h->device) ||
        h->n > symv_max_n()) {
      set_error("vie_assemble: VIE_OPERATOR_SYM32 needs the displacement kernel, its expansion and the "
                "block product (2D, FP32 tiles, S = 64, n <= 160)");
      return VIE_ERR_UNSUPPORTED;
    }
    if (!reuse) VIE_CUDA(vie_malloc(&h->kmat, sizeof(float) * symv_block_floats(h->n)));
    if (!h->sym_partial) VIE_CUDA(vie_malloc((void **)&h->sym_partial, sizeof(float) * symv_partial_floats(h->n)));
    if (!h->pairs) VIE_CUDA(vie_malloc(&h->pairs, sizeof(float) * (size_t)h->disp.stored));
    const double hh = 1.0 / h->n;
    const float tau_scale2 = (float)(hh / h->opts.steps * 1.4426950408889634);
    const float wcoef = (float)(hh / (2.0 * kPi));
    vie_status s = disp_store(h->disp, h->n, tau_scale2, wcoef, (float *)h->pairs, st);
    if (s != VIE_OK) return s;
    s = disp_expand(h->disp, h->n, (const float *)h->pairs, h->sig_s, h->diag, 0, (float *)h->kmat, nullptr,
                    nullptr, h->device, st);
    if (s != VIE_OK) return s;
    h->asm_mode = mode;
    return VIE_OK;
  }
  if (mode == VIE_OPERATOR_PAIRS32) {
    // every unordered pair's FP32 weight, displacement-major (the displacement kernel's march)
    if (h->use_kernel != VIE_KERNEL_DISPLACEMENT || h->dim != 2) {
      set_error("vie_assemble: VIE_OPERATOR_PAIRS32 needs the displacement kernel (2D, FP32 tiles, S = 64, "
                "n <= 258)");
      return VIE_ERR_UNSUPPORTED;
    }
    if (!reuse) VIE_CUDA(vie_malloc(&h->kmat, sizeof(float) * (size_t)h->disp.stored));
    const double hh = 1.0 / h->n;
    const float tau_scale2 = (float)(hh / h->opts.steps * 1.4426950408889634);
    const float wcoef = (float)(hh / (2.0 * kPi));
    vie_status s = disp_store(h->disp, h->n, tau_scale2, wcoef, (float *)h->kmat, st);
    if (s != VIE_OK) return s;
    h->asm_mode = mode;
    return VIE_OK;
  }
  // dense K from the displacement kernel's pair weights where the expansion
  // has room for the grid, else from the tile-pair assembler (M-iii only)
  const bool disp2 =
      h->use_kernel == VIE_KERNEL_DISPLACEMENT && h->dim == 2 && disp_expand_fits(h->n, h->device);
  // 3D: the pair weights of the 3D displacement kernel, expanded along grid lines
  const bool disp3 = h->use_kernel == VIE_KERNEL_DISPLACEMENT && h->dim == 3 && h->disp3.usable &&
                     h->opts.disc == VIE_DISC_MIII;
  if (!disp2 && h->opts.disc == VIE_DISC_MII) {
    set_error("vie_assemble: dense K with VIE_DISC_MII needs the pair-weight expansion (n <= 169)");
    return VIE_ERR_UNSUPPORTED;
  }
  if ((!h->sym.usable && !disp2 && !disp3) || h->opts.precision != VIE_PREC_FP32 ||
      h->opts.tau_mode != VIE_TAU_MARCH || h->opts.steps != 64) {
    set_error("vie_assemble: needs FP32 tiles, the march, S = 64 and a grid whose sigma_t fits "
              "in shared memory");
    return VIE_ERR_UNSUPPORTED;
  }
  const long N = h->N;
  h->ldk = assembled_ldk(N);
  const size_t half = sizeof(short) * (size_t)N * h->ldk;
  vie_status s;
  if (reuse) {
    // same storage, entries recomputed in place
  } else if (mode == VIE_OPERATOR_FP32) {
    VIE_CUDA(vie_malloc(&h->kmat, 2 * half));
  } else {
    VIE_CUDA(vie_malloc(&h->kmat, half));
    cudaError_t e = vie_malloc(&h->kmat_lo, half);
    if (e != cudaSuccess) {
      vie_free(h->kmat);
      h->kmat = nullptr;
      return cuda_fail(e, "cudaMalloc");
    }
  }
  if (!h->dev_err && (s = dalloc(&h->dev_err, 1)) != VIE_OK) return s;
  VIE_CUDA(cudaMemsetAsync(h->dev_err, 0, sizeof(int), st));
  float *k32 = mode == VIE_OPERATOR_FP32 ? (float *)h->kmat : nullptr;
  void *khi = mode == VIE_OPERATOR_BF16X3 ? h->kmat : nullptr;
  if (disp2) {
    // march every unordered pair once into the pair weights, then expand them into K
    if (!h->pairs) VIE_CUDA(vie_malloc(&h->pairs, sizeof(float) * (size_t)h->disp.stored));
    const double hh = 1.0 / h->n;
    const float tau_scale2 = (float)(hh / h->opts.steps * 1.4426950408889634);
    const float wcoef = (float)(hh / (2.0 * kPi));
    s = disp_store(h->disp, h->n, tau_scale2, wcoef, (float *)h->pairs, st);
    if (s != VIE_OK) return s;
    s = disp_expand(h->disp, h->n, (const float *)h->pairs, h->sig_s, h->diag, h->ldk, k32, khi, h->kmat_lo,
                    h->device, st);
  } else if (disp3) {
    const double hh = 1.0 / h->n;
    s = disp3_assemble(&h->disp3, (float)(hh / h->opts.steps * 1.4426950408889634), (float)(hh / (4.0 * kPi)),
                       h->sig_s, h->diag, h->ldk, k32, khi, h->kmat_lo, h->device, st);
  } else {
    s = launch_assemble(h->sym, h->dim, h->n, N, h->sig_s, h->diag, k32, khi, h->kmat_lo, h->device, st);
  }
  if (s != VIE_OK) return s;
  h->asm_mode = mode;
  return VIE_OK;
}

vie_status vie_assemble(vie_handle *h, int mode, void *stream) { return assemble_impl(h, mode, 6, stream); }

vie_status vie_assemble_fmm(vie_handle *h, int order, void *stream) {
  return assemble_impl(h, VIE_OPERATOR_FMM, order, stream);
}

vie_status vie_set_preconditioner(vie_handle *h, vie_unet *u, double s_ref) {
  if (!h) return invalid("vie_set_preconditioner: NULL handle");
  if (!u) {
    h->precond = nullptr;
    return VIE_OK;
  }
  if (h->dim != 2) return invalid("vie_set_preconditioner: 2D handles only");
  if (!(s_ref > 0.0)) return invalid("vie_set_preconditioner: s_ref must be > 0");
  const int levels = unet_levels(u);
  if (h->n % (1 << (levels - 1)) != 0)
    return invalid("vie_set_preconditioner: n must be divisible by 2^(levels-1)");
  h->precond = unet_impl(u);
  h->precond_inv_ref = 1.0 / s_ref;
  h->precond_on_diff = false;
  fft_release(&h->fft);  // one preconditioner at a time
  diffusion_release(&h->diff);
  return VIE_OK;
}

vie_status vie_set_preconditioner_on_diffusion(vie_handle *h, vie_unet *u, double s_ref, void *stream) {
  if (!h) return invalid("vie_set_preconditioner_on_diffusion: NULL handle");
  if (!u) {
    h->precond = nullptr;
    h->precond_on_diff = false;
    diffusion_release(&h->diff);
    return VIE_OK;
  }
  vie_status s = vie_set_preconditioner(h, u, s_ref);
  if (s != VIE_OK) return s;
  UnetImpl *net = h->precond;
  const double inv = h->precond_inv_ref;
  if ((s = vie_set_diffusion_preconditioner(h, 1, stream)) != VIE_OK) return s;  // clears the network
  h->precond = net;
  h->precond_inv_ref = inv;
  h->precond_on_diff = true;
  return VIE_OK;
}

vie_status vie_set_fft_preconditioner(vie_handle *h, int enable, void *stream) {
  if (!h) return invalid("vie_set_fft_preconditioner: NULL handle");
  DeviceGuard dg(h->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  if (!enable) {
    VIE_CUDA(cudaStreamSynchronize(st));
    fft_release(&h->fft);
    return VIE_OK;
  }
  if (h->dim != 2) return invalid("vie_set_fft_preconditioner: 2D handles only");
  // the mean coefficients of the medium (Section 4.4: mu -> its mean over Omega)
  std::vector<double> t((size_t)h->N), ss((size_t)h->N);
  VIE_CUDA(cudaMemcpy(t.data(), h->sig_t, sizeof(double) * h->N, cudaMemcpyDeviceToHost));
  VIE_CUDA(cudaMemcpy(ss.data(), h->sig_s, sizeof(double) * h->N, cudaMemcpyDeviceToHost));
  double mu = 0.0, mu_s = 0.0;
  for (long i = 0; i < h->N; ++i) {
    mu += t[i];
    mu_s += ss[i];
  }
  mu /= (double)h->N;
  mu_s /= (double)h->N;
  VIE_CUDA(cudaStreamSynchronize(st));
  vie_status s = fft_prepare(&h->fft, h->n, mu, mu_s, h->opts.disc == VIE_DISC_MII, st);
  if (s != VIE_OK) return s;
  h->precond = nullptr;  // one preconditioner at a time
  diffusion_release(&h->diff);
  return VIE_OK;
}

vie_status vie_set_diffusion_preconditioner(vie_handle *h, int enable, void *stream) {
  if (!h) return invalid("vie_set_diffusion_preconditioner: NULL handle");
  DeviceGuard dg(h->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  VIE_CUDA(cudaStreamSynchronize(st));
  if (!enable) {
    diffusion_release(&h->diff);
    return VIE_OK;
  }
  if (h->dim != 2) return invalid("vie_set_diffusion_preconditioner: 2D handles only");
  std::vector<double> t((size_t)h->N), ss((size_t)h->N);
  VIE_CUDA(cudaMemcpy(t.data(), h->sig_t, sizeof(double) * h->N, cudaMemcpyDeviceToHost));
  VIE_CUDA(cudaMemcpy(ss.data(), h->sig_s, sizeof(double) * h->N, cudaMemcpyDeviceToHost));
  vie_status s = diffusion_prepare(&h->diff, h->n, t.data(), ss.data(), h->sig_s, st);
  if (s != VIE_OK) {
    diffusion_release(&h->diff);
    return s;
  }
  h->precond = nullptr;  // one preconditioner at a time
  h->precond_on_diff = false;
  fft_release(&h->fft);
  return VIE_OK;
}

vie_status vie_diffusion_precondition(vie_handle *h, const double *v, double *z, void *stream) {
  if (!h || !v || !z) return invalid("vie_diffusion_precondition: NULL argument");
  if (!h->diff.on)
    return invalid("vie_diffusion_precondition: no diffusion preconditioner (vie_set_diffusion_preconditioner)");
  DeviceGuard dg(h->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const long N = h->N;
  const bool vd = is_device_ptr(v), zd = is_device_ptr(z);
  const double *vv = v;
  double *zz = z;
  vie_status s;
  if (!vd) {
    if ((s = h->stage_a.reserve(N)) != VIE_OK) return s;
    VIE_CUDA(cudaMemcpyAsync(h->stage_a.ptr, v, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    vv = h->stage_a.ptr;
  }
  if (!zd) {
    if ((s = h->stage_b.reserve(N)) != VIE_OK) return s;
    zz = h->stage_b.ptr;
  }
  if ((s = diffusion_precondition(h->diff, vv, zz, st)) != VIE_OK) return s;
  if (!zd) {
    VIE_CUDA(cudaMemcpyAsync(z, zz, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    VIE_CUDA(cudaStreamSynchronize(st));
  }
  return VIE_OK;
}

vie_status vie_fft_precondition(vie_handle *h, const double *v, double *z, void *stream) {
  if (!h || !v || !z) return invalid("vie_fft_precondition: NULL argument");
  if (!h->fft.on) return invalid("vie_fft_precondition: no FFT preconditioner (vie_set_fft_preconditioner)");
  DeviceGuard dg(h->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const long N = h->N;
  const bool vd = is_device_ptr(v), zd = is_device_ptr(z);
  const double *vv = v;
  double *zz = z;
  vie_status s;
  if (!vd) {
    if ((s = h->stage_a.reserve(N)) != VIE_OK) return s;
    VIE_CUDA(cudaMemcpyAsync(h->stage_a.ptr, v, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    vv = h->stage_a.ptr;
  }
  if (!zd) {
    if ((s = h->stage_b.reserve(N)) != VIE_OK) return s;
    zz = h->stage_b.ptr;
  }
  if ((s = fft_precondition(h->fft, vv, zz, st)) != VIE_OK) return s;
  if (!zd) {
    VIE_CUDA(cudaMemcpyAsync(z, zz, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
    VIE_CUDA(cudaStreamSynchronize(st));
  }
  return VIE_OK;
}

vie_status vie_solve_gmres(vie_handle *h, const double *f, double *U, const vie_gmres_opts *o,
                           vie_report *rep, void *stream) {
  if (!h || !f || !U) return invalid("vie_solve_gmres: NULL argument");
  vie_gmres_opts opt;
  vie_default_gmres_opts(&opt);
  if (o) opt = *o;
  if (!(opt.rtol > 0.0) || opt.restart < 1 || opt.restart > 256 || opt.maxit < 1)
    return invalid("vie_solve_gmres: rtol > 0, 1 <= restart <= 256, maxit >= 1 required");
  if (opt.nrhs < 1 || opt.nrhs > 4096) return invalid("vie_solve_gmres: 1 <= nrhs <= 4096 required");
  DeviceGuard dg(h->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  auto t_start = std::chrono::steady_clock::now();
  cudaStream_t st = (cudaStream_t)stream;
  const long N = h->N;
  const int m = opt.restart;
  vie_status s;
  if (opt.nrhs > 1) {
    // several sources on this medium: lockstep solves
    const int R = opt.nrhs;
    const size_t total = (size_t)R * N;
    h->t_apply_ms = h->t_kernel_ms = 0.0;
    h->n_apply = 0;
    const bool fd = is_device_ptr(f), ud = is_device_ptr(U);
    const double *fdev = f;
    double *x = U;
    if (!fd) {
      if ((s = h->stage_a.reserve(total)) != VIE_OK) return s;
      VIE_CUDA(cudaMemcpyAsync(h->stage_a.ptr, f, sizeof(double) * total, cudaMemcpyHostToDevice, st));
      fdev = h->stage_a.ptr;
    }
    if (!ud) {
      if ((s = h->stage_b.reserve(total)) != VIE_OK) return s;
      x = h->stage_b.ptr;
      if (!opt.zero_x0) VIE_CUDA(cudaMemcpyAsync(x, U, sizeof(double) * total, cudaMemcpyHostToDevice, st));
    }
    if (opt.zero_x0) VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * total, st));
    s = solve_multi(h, fdev, x, R, opt, rep, st, opt.time_apply != 0, t_start);
    if (s != VIE_OK && s != VIE_ERR_NOT_CONVERGED) return s;
    if (!ud) {
      VIE_CUDA(cudaMemcpyAsync(U, x, sizeof(double) * total, cudaMemcpyDeviceToHost, st));
      VIE_CUDA(cudaStreamSynchronize(st));
    }
    return s;
  }
  if ((s = ensure_gmres(h, m)) != VIE_OK) return s;
  const bool has_precond = h->precond || h->fft.on || h->diff.on;
  if (has_precond && h->z_m < m) {
    dfree(h->Z);
    if ((s = dalloc(&h->Z, (size_t)m * N)) != VIE_OK) return s;
    h->z_m = m;
  }
  if (h->precond && !h->net_x && (s = dalloc(&h->net_x, (size_t)3 * N)) != VIE_OK) return s;
  h->t_apply_ms = h->t_kernel_ms = 0.0;
  h->n_apply = 0;
  const bool timed = opt.time_apply != 0;
  const bool fd = is_device_ptr(f), ud = is_device_ptr(U);
  const double *fdev = f;
  double *x = U;
  if (!fd) {
    if ((s = h->stage_a.reserve(N)) != VIE_OK) return s;
    VIE_CUDA(cudaMemcpyAsync(h->stage_a.ptr, f, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    fdev = h->stage_a.ptr;
  }
  if (!ud) {
    if ((s = h->stage_b.reserve(N)) != VIE_OK) return s;
    x = h->stage_b.ptr;
    if (!opt.zero_x0)
      VIE_CUDA(cudaMemcpyAsync(x, U, sizeof(double) * N, cudaMemcpyHostToDevice, st));
  }
  if (opt.zero_x0) VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, st));
  // phi = A f (Eq. EQ:ERT Intgrl FMM), unless the caller passed phi.
  if (opt.rhs_is_phi) {
    VIE_CUDA(cudaMemcpyAsync(h->phi, fdev, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
  } else if ((s = apply_dev(h, VIE_OP_A_RAW, fdev, h->phi, st, timed)) != VIE_OK) {
    return s;
  }
  double bn2 = 0.0;
  if ((s = norm2_dev(h, h->phi, h->scal, st)) != VIE_OK) return s;
  if ((s = read_scalar(h, h->scal, &bn2, st)) != VIE_OK) return s;
  if (!isfinite(bn2)) {
    set_error("vie_solve_gmres: non-finite right-hand side");
    return VIE_ERR_NONFINITE;
  }
  const double bnorm = sqrt(bn2);
  vie_report R{};
  R.relres = 0.0;
  R.relres_est = 0.0;
  bool converged = false;
  if (bnorm == 0.0) {
    VIE_CUDA(cudaMemsetAsync(x, 0, sizeof(double) * N, st));
    converged = true;
  }
  const int blocks = dot_blocks(N);
  bool x_is_zero = opt.zero_x0 != 0;
  while (!converged) {
    // true residual r = phi - (I - K) x
    if (x_is_zero) {
      VIE_CUDA(cudaMemcpyAsync(h->r, h->phi, sizeof(double) * N, cudaMemcpyDeviceToDevice, st));
    } else {
      if ((s = apply_dev(h, VIE_OP_I_MINUS_K, x, h->w, st, timed)) != VIE_OK) return s;
      if ((s = launch_axpby(1.0, h->phi, -1.0, h->w, h->r, N, st)) != VIE_OK) return s;
    }
    x_is_zero = false;
    double rn2 = 0.0;
    if ((s = norm2_dev(h, h->r, h->scal + 1, st)) != VIE_OK) return s;
    if ((s = read_scalar(h, h->scal + 1, &rn2, st)) != VIE_OK) return s;
    if (!isfinite(rn2)) {
      set_error("vie_solve_gmres: non-finite residual");
      return VIE_ERR_NONFINITE;
    }
    const double beta = sqrt(rn2);
    R.relres = beta / bnorm;
    if (R.relres <= opt.rtol) {
      converged = true;
      break;
    }
    if (R.iters >= opt.maxit) break;
    // V_0 = r / beta, gv = beta e_1
    if ((s = launch_scale(h->r, h->scal + 1, 1, h->V, N, st)) != VIE_OK) return s;
    for (int i = 0; i <= m; ++i) h->h_pinned[i] = 0.0;
    h->h_pinned[0] = beta;
    VIE_CUDA(cudaMemcpyAsync(h->gv, h->h_pinned, sizeof(double) * (m + 1), cudaMemcpyHostToDevice, st));
    int k = 0;
    const bool flexible = has_precond && !R.fell_back;
    double est_prev = 1e300, est_prev2 = 1e300;
    bool stall = false;
    while (k < m && R.iters < opt.maxit) {
      double *vk = h->V + (size_t)k * N;
      double *vk1 = h->V + (size_t)(k + 1) * N;
      const double *op_in = vk;
      if (flexible) {
        // z_k = M(v_k) (right preconditioning, flexible GMRES)
        double *zk = h->Z + (size_t)k * N;
        if (h->fft.on) {
          // the FFT preconditioner (Section 4.4, Eq. EQ:SOL FFT)
          if ((s = fft_precondition(h->fft, vk, zk, st)) != VIE_OK) return s;
        } else if (h->precond && h->precond_on_diff) {
          // the diffusion preconditioner, then the network's correction of it
          if ((s = diffusion_precondition(h->diff, vk, zk, st)) != VIE_OK) return s;
          if ((s = norm2_dev(h, vk, h->scal + 4, st)) != VIE_OK) return s;
          if ((s = unet_precondition(h->precond, h->sig_t, h->sig_s, h->precond_inv_ref, vk, h->scal + 4,
                                     h->n, h->net_x, zk, zk, st)) != VIE_OK)
            return s;
        } else if (h->diff.on) {
          // the diffusion preconditioner (Section 4.4, Eq. EQ:DA)
          if ((s = diffusion_precondition(h->diff, vk, zk, st)) != VIE_OK) return s;
        } else {
          if ((s = norm2_dev(h, vk, h->scal + 4, st)) != VIE_OK) return s;
          if ((s = unet_precondition(h->precond, h->sig_t, h->sig_s, h->precond_inv_ref, vk, h->scal + 4,
                                     h->n, h->net_x, nullptr, zk, st)) != VIE_OK)
            return s;
        }
        op_in = zk;
        ++R.precond_iters;
      }
      if ((s = apply_dev(h, VIE_OP_I_MINUS_K, op_in, vk1, st, timed)) != VIE_OK) return s;
      // CGS2: two passes of h = V^T w, w -= V h; hcol accumulates both.
      // (each dot pass is one launch: its last block sums the block partials)
      if ((s = launch_dots_last(h->V, k + 1, N, vk1, N, h->part, blocks, h->ticket, h->hcol, nullptr, st)) !=
          VIE_OK)
        return s;
      if ((s = launch_orth_update(h->V, k + 1, N, h->hcol, vk1, N, st)) != VIE_OK) return s;
      if ((s = launch_dots_last(h->V, k + 1, N, vk1, N, h->part, blocks, h->ticket, h->htmp, h->hcol, st)) !=
          VIE_OK)
        return s;
      if ((s = launch_orth_update(h->V, k + 1, N, h->htmp, vk1, N, st)) != VIE_OK) return s;
      if ((s = launch_norm2_givens(vk1, N, h->part, blocks, h->ticket, h->scal + 2, h->H, m, k, h->hcol, h->cs,
                                   h->sn, h->gv, bnorm, h->scal + 3, st)) != VIE_OK)
        return s;
      if ((s = launch_scale(vk1, h->scal + 2, 1, vk1, N, st)) != VIE_OK) return s;
      double est = 0.0;
      if ((s = read_scalar(h, h->scal + 3, &est, st)) != VIE_OK) return s;
      if (timed && (s = harvest_events(h)) != VIE_OK) return s;
      ++k;
      ++R.iters;
      R.relres_est = est;
      if (!isfinite(est)) {
        if (flexible) {
          // the preconditioner produced a non-finite direction: drop this step
          --k;
          stall = true;
          break;
        }
        set_error("vie_solve_gmres: non-finite Arnoldi step");
        return VIE_ERR_NONFINITE;
      }
      if (est <= opt.rtol) break;
      if (flexible && k >= 2 && est > 0.8 * est_prev && est_prev > 0.8 * est_prev2) {
        stall = true;
        break;
      }
      est_prev2 = est_prev;
      est_prev = est;
    }
    if (k > 0) {
      if ((s = launch_backsolve(h->H, m, k, h->gv, h->yv, st)) != VIE_OK) return s;
      if ((s = launch_lincomb_add(flexible ? h->Z : h->V, k, N, h->yv, x, N, st)) != VIE_OK) return s;
    }
    if (stall) R.fell_back = 1;
    ++R.restarts;
  }
  if (!ud) VIE_CUDA(cudaMemcpyAsync(U, x, sizeof(double) * N, cudaMemcpyDeviceToHost, st));
  VIE_CUDA(cudaStreamSynchronize(st));
  if (timed && (s = harvest_events(h)) != VIE_OK) return s;
  R.converged = converged ? 1 : 0;
  R.n_apply = h->n_apply;
  R.t_apply_ms = h->t_apply_ms;
  R.t_apply_kernel_ms = h->t_kernel_ms;
  R.t_total_ms =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t_start).count();
  if (rep) *rep = R;
  if (!converged) {
    set_error("vie_solve_gmres: maxit reached before rtol");
    return VIE_ERR_NOT_CONVERGED;
  }
  return VIE_OK;
}

vie_status ert_sweep(vie_handle *h, const double *U, const double *f, const float *dirs, int M,
                     float *Phi, void *stream) {
  if (!h || !U || !f || !dirs || !Phi) return invalid("ert_sweep: NULL argument");
  if (M < 1) return invalid("ert_sweep: M must be >= 1");
  DeviceGuard dg(h->device);
  if (dg.err != cudaSuccess) return cuda_fail(dg.err, "cudaSetDevice");
  cudaStream_t st = (cudaStream_t)stream;
  const long N = h->N;
  vie_status s;
  const double *Ud = U, *fd = f;
  const float *dd = dirs;
  float *Pd = Phi;
  if (!is_device_ptr(U)) {
    if ((s = h->stage_a.reserve(N)) != VIE_OK) return s;
    VIE_CUDA(cudaMemcpyAsync(h->stage_a.ptr, U, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    Ud = h->stage_a.ptr;
  }
  if (!is_device_ptr(f)) {
    if ((s = h->stage_c.reserve(N)) != VIE_OK) return s;
    VIE_CUDA(cudaMemcpyAsync(h->stage_c.ptr, f, sizeof(double) * N, cudaMemcpyHostToDevice, st));
    fd = h->stage_c.ptr;
  }
  if (!is_device_ptr(dirs)) {
    for (int m = 0; m < M; ++m) {
      double n2 = 0.0;
      for (int d = 0; d < h->dim; ++d) n2 += (double)dirs[m * h->dim + d] * dirs[m * h->dim + d];
      if (!(fabs(n2 - 1.0) < 1e-5)) return invalid("ert_sweep: directions must be unit vectors");
    }
    if ((s = h->stage_f1.reserve((size_t)M * h->dim)) != VIE_OK) return s;
    VIE_CUDA(cudaMemcpyAsync(h->stage_f1.ptr, dirs, sizeof(float) * M * h->dim,
                             cudaMemcpyHostToDevice, st));
    dd = h->stage_f1.ptr;
  }
  const bool pd = is_device_ptr(Phi);
  if (!pd) {
    if ((s = h->stage_f2.reserve((size_t)M * N)) != VIE_OK) return s;
    Pd = h->stage_f2.ptr;
  }
  if (!h->qpad) {
    const long lattice = h->dim == 2 ? (long)h->P * h->P : (long)h->P * h->P * h->P;
    if ((s = dalloc(&h->qpad, lattice)) != VIE_OK) return s;
  }
  if ((s = launch_make_q(h->dim, h->n, h->sig_s, Ud, fd, h->qpad, st)) != VIE_OK) return s;
  if ((s = launch_sweep(h->dim, h->n, h->sig32, h->qpad, dd, M, Pd, st)) != VIE_OK) return s;
  if (!pd) {
    VIE_CUDA(cudaMemcpyAsync(Phi, Pd, sizeof(float) * M * N, cudaMemcpyDeviceToHost, st));
    VIE_CUDA(cudaStreamSynchronize(st));
  }
  return VIE_OK;
}

}  // extern "C"
