// Host side of libs3ttv: argument checks, device workspace, the per-pass launch
// sequence of Alg. 1 and the C ABI declared in include/s3ttv.h.
#include <chrono>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "s3ttv.h"
#include "s3ttv_internal.cuh"

using namespace s3ttv;

struct s3ttv_ctx {
  int device = 0;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  int num_sms = 0;
  char err[512] = {0};
  // options
  int step_policy = S3TTV_STEP_PAPER;
  int check_every = 16;
  int jacobi_max_sweeps = 24;
  float jacobi_tol = 1e-4f;   // a sweep with no pair above it ends an eigen-solve
  float jacobi_polish = 0.f;  // 0: the default, kDefaultPolish (jacobi_polish_for)
  float first_order = 0.f;  // remainder bound of the first-order clip (0: off, the default)
  int batch_worklist = 0;    // batched solves: 1, one block-dual work list per block side
  int tensor_cores = 2;  // block-dual form: 2 streaming (tensor cores), 1 group (tensor cores), 0 CUDA cores
  int layout = S3TTV_LAYOUT_PAPER;  // block matrices: paper k^2 x 2N3 or stacked 2k^2 x N3
  int open_s = 0;                   // 1: D_s stops at the last band (no wrap-around)
  int reg = S3TTV_REG_S3TTV;        // regularisation function (S3TTV or a comparison method)
  float hsstv_omega = 0.05f;        // HSSTV's weight of the first-order differences
  int autotune = 0;                 // 1: time the block-dual forms on the first passes, keep the fastest
  int tuned_tc = -1, tuned_minb = 0;  // the chosen form (tc -1: none chosen yet)
  int tuned_k = 0, tuned_n3p = 0;     // the problem shape it was chosen for
  // problem
  bool ready = false;
  Dims dm{};
  int k = 0;
  float eps = 0.f, alpha = 0.f, beta = 0.f, mu_min = 0.f, mu_max = 1.f;
  double gam[6] = {0, 0, 0, 0, 0, 0};
  int parity = 0;  // which of t[2], Zv[2], Zh[2] holds the current value
  // device workspace
  size_t cap_np = 0, cap_y = 0, cap_stage = 0, cap_w = 0;
  float *v = nullptr, *u = nullptr, *s = nullptr, *t[2] = {nullptr, nullptr}, *y2 = nullptr, *d = nullptr;
  float *ubar = nullptr, *zs = nullptr, *zt = nullptr, *Zv[2] = {nullptr, nullptr}, *Zh[2] = {nullptr, nullptr};
  float *Fv = nullptr, *Fh = nullptr;  // D_v D_s ubar, D_h D_s ubar
  float *Fs = nullptr, *Zs[2] = {nullptr, nullptr};  // SSST: D_s ubar and the third part of Z
  int *fb_list = nullptr;  // FP64 re-solve queue of the block duals
  int fb_cap = 0;
  bool fp64_fallback = true;  // option
  size_t alloc_limit = 0;     // option: device bytes the context may hold (0: no limit)
  bool nvtx = false;          // option: NVTX ranges around calls and kernel classes
  float *Y = nullptr, *stage = nullptr;
  float *W = nullptr;      // per-block warm-start rows of the eigen-solve
  long long w_stride = 0;
  bool warm_valid = false; // W holds the rows of the current Y
  bool warm_start = true;  // option
  Scalars *sc = nullptr;
  double *part = nullptr;  // [3][kMaxGrid]
  unsigned *hcnt = nullptr;
  double *hsum = nullptr;
  double *macc = nullptr;  // accumulators of s3ttv_quality / s3ttv_objective
  size_t cap_macc = 0;
  size_t bytes = 0;
  // launch accounting and optional per-class event timing
  long long launches = 0;
  bool profile = false;
  cudaEvent_t *ev = nullptr;  // [6 * ev_passes]
  int ev_passes = 0;
  double prof_ms[S3TTV_KERNEL_CLASSES] = {0, 0, 0, 0, 0};
  long long prof_n[S3TTV_KERNEL_CLASSES] = {0, 0, 0, 0, 0};
  // batched solves: one member context (workspace and stream) per problem
  std::vector<s3ttv_ctx *> members;
  BatchDual *batch_items = nullptr;  // the block-dual work lists of a batched solve (device)
  size_t cap_items = 0;
  float *rows = nullptr;  // blocks above 12 x 12: the per-CTA n x n matrices of the block duals
  size_t cap_rows = 0;    // bytes
};

namespace {

constexpr int kMaxGrid = 4096;
constexpr int kMaxK = kMaxLargeK;  // k <= 5: block_dual.cu; 6..16: block_dual_large.cu
constexpr int kLaunchesPerPass = 10;  // kernels enqueue_pass launches (block-dual regularisers, no re-solve)
constexpr int kFbQueueMax = 1 << 16;  // entries of the FP64 re-solve queue

int fail(s3ttv_ctx *c, int status, const char *fmt, ...) {
  if (c) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(c->err, sizeof(c->err), fmt, ap);
    va_end(ap);
  }
  return status;
}

#define CU(call)                                                                            \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return fail(ctx, S3TTV_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));         \
  } while (0)

struct DeviceGuard {
  int prev = -1;
  explicit DeviceGuard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~DeviceGuard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool is_device_ptr(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int round4(int x) { return (x + 3) & ~3; }

// NVTX ranges (option S3TTV_OPT_NVTX): one per API call, and one per kernel
// class as a pass is enqueued, so a profiler can attribute launches to the steps
// of Alg. 1.  No-ops unless the option is on (and cheap without a tool attached).
struct NvtxRange {
  bool on;
  NvtxRange(bool enable, const char *name) : on(enable) {
    if (on) nvtxRangePushA(name);
  }
  ~NvtxRange() {
    if (on) nvtxRangePop();
  }
};
struct NvtxPhase {  // consecutive ranges: next() closes the open one
  bool on, open = false;
  explicit NvtxPhase(bool enable) : on(enable) {}
  void next(const char *name) {
    if (!on) return;
    if (open) nvtxRangePop();
    nvtxRangePushA(name);
    open = true;
  }
  ~NvtxPhase() {
    if (open) nvtxRangePop();
  }
};

bool is_hsstv(const s3ttv_ctx *c) { return c->reg == S3TTV_REG_HSSTV1 || c->reg == S3TTV_REG_HSSTV2; }
bool is_ssst(const s3ttv_ctx *c) { return c->reg == S3TTV_REG_SSST; }
// parts of a block row: [D_v | D_h] (S3TTV, STV) or SSST's [D_v | D_h | D_s]
int row_parts(const s3ttv_ctx *c) { return is_ssst(c) ? 3 : 2; }

int elementwise_grid(const s3ttv_ctx *c, long long n) {
  long long g = (n + 255) / 256;
  long long cap = (long long)c->num_sms * 8;
  if (cap > kMaxGrid) cap = kMaxGrid;
  if (g > cap) g = cap;
  if (g < 1) g = 1;
  return (int)g;
}

void free_all(s3ttv_ctx *c) {
  float **bufs[] = {&c->v, &c->u, &c->s, &c->t[0], &c->t[1], &c->y2, &c->d, &c->ubar, &c->zs,
                    &c->zt, &c->Zv[0], &c->Zv[1], &c->Zh[0], &c->Zh[1], &c->Y, &c->stage, &c->W,
                    &c->Fv, &c->Fh, &c->Fs, &c->Zs[0], &c->Zs[1]};
  for (float **b : bufs) {
    if (*b) cudaFree(*b);
    *b = nullptr;
  }
  if (c->sc) cudaFree(c->sc);
  if (c->fb_list) cudaFree(c->fb_list);
  c->fb_list = nullptr;
  c->fb_cap = 0;
  if (c->part) cudaFree(c->part);
  if (c->hcnt) cudaFree(c->hcnt);
  if (c->hsum) cudaFree(c->hsum);
  if (c->macc) cudaFree(c->macc);
  if (c->batch_items) cudaFree(c->batch_items);
  c->batch_items = nullptr;
  c->cap_items = 0;
  if (c->rows) cudaFree(c->rows);
  c->rows = nullptr;
  c->cap_rows = 0;
  c->macc = nullptr;
  c->cap_macc = 0;
  c->sc = nullptr;
  c->part = nullptr;
  c->hcnt = nullptr;
  c->hsum = nullptr;
  c->cap_np = c->cap_y = c->cap_stage = c->cap_w = 0;
  c->bytes = 0;
  c->ready = false;
  c->warm_valid = false;
}

int dmalloc(s3ttv_ctx *ctx, void **p, size_t bytes) {
  if (ctx->alloc_limit && ctx->bytes + bytes > ctx->alloc_limit) {
    *p = nullptr;
    return fail(ctx, S3TTV_ENOMEM, "allocating %zu bytes would pass the context's limit of %zu (holding %zu)", bytes,
                ctx->alloc_limit, ctx->bytes);
  }
  cudaError_t e = cudaMalloc(p, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    *p = nullptr;
    return fail(ctx, S3TTV_ENOMEM, "cudaMalloc of %zu bytes failed: %s", bytes, cudaGetErrorString(e));
  }
  ctx->bytes += bytes;
  return S3TTV_OK;
}

// Small buffers every entry point needs.
int ensure_common(s3ttv_ctx *ctx) {
  if (ctx->sc) return S3TTV_OK;
  int rc;
  if ((rc = dmalloc(ctx, (void **)&ctx->sc, sizeof(Scalars)))) return rc;
  if ((rc = dmalloc(ctx, (void **)&ctx->part, sizeof(double) * 3 * kMaxGrid))) return rc;
  if ((rc = dmalloc(ctx, (void **)&ctx->hcnt, sizeof(unsigned) * 2 * kHistBins))) return rc;
  if ((rc = dmalloc(ctx, (void **)&ctx->hsum, sizeof(double) * 2 * kHistBins))) return rc;
  CU(cudaMemsetAsync(ctx->hcnt, 0, sizeof(unsigned) * 2 * kHistBins, ctx->stream));
  CU(cudaMemsetAsync(ctx->hsum, 0, sizeof(double) * 2 * kHistBins, ctx->stream));
  return S3TTV_OK;
}

int ensure_stage(s3ttv_ctx *ctx, size_t elems) {
  if (elems <= ctx->cap_stage) return S3TTV_OK;
  if (ctx->stage) {
    cudaFree(ctx->stage);
    ctx->bytes -= ctx->cap_stage * sizeof(float);
    ctx->stage = nullptr;
    ctx->cap_stage = 0;
  }
  int rc = dmalloc(ctx, (void **)&ctx->stage, elems * sizeof(float));
  if (rc) return rc;
  ctx->cap_stage = elems;
  return S3TTV_OK;
}

// Problem-sized buffers; reuses them when they are large enough.
int ensure_macc(s3ttv_ctx *ctx, size_t n) {
  if (n <= ctx->cap_macc) return S3TTV_OK;
  if (ctx->macc) {
    cudaFree(ctx->macc);
    ctx->bytes -= ctx->cap_macc * sizeof(double);
    ctx->macc = nullptr;
    ctx->cap_macc = 0;
  }
  int rc = dmalloc(ctx, (void **)&ctx->macc, n * sizeof(double));
  if (rc) return rc;
  ctx->cap_macc = n;
  return S3TTV_OK;
}

int ensure_problem_buffers(s3ttv_ctx *ctx, const Dims &dm, int k) {
  const size_t np = (size_t)dm.Np;
  size_t ny = (size_t)dm.P * k * k * row_parts(ctx) * dm.N3p;
  if (ny < 4 * np) ny = 4 * np;  // HSSTV keeps four dual cubes
  const long long ws = ctx->layout == S3TTV_LAYOUT_STACKED ? block_dual_large_w_stride(k, true)
                       : is_ssst(ctx)                      ? block_dual_large_w_stride(k, false)
                                                           : block_dual_w_stride(k);
  const size_t nw = (size_t)dm.P * ws;
  ctx->w_stride = ws;
  const int want_fb = dm.P < kFbQueueMax ? (int)dm.P : kFbQueueMax;
  if (np <= ctx->cap_np && ny <= ctx->cap_y && nw <= ctx->cap_w && ctx->sc && (!is_ssst(ctx) || ctx->Fs) &&
      want_fb <= ctx->fb_cap)
    return S3TTV_OK;
  free_all(ctx);
  ctx->w_stride = ws;
  int rc = ensure_common(ctx);
  if (rc) return rc;
  float **cubes[] = {&ctx->v, &ctx->u, &ctx->s, &ctx->t[0], &ctx->t[1], &ctx->y2, &ctx->d, &ctx->ubar,
                     &ctx->zs, &ctx->zt, &ctx->Zv[0], &ctx->Zv[1], &ctx->Zh[0], &ctx->Zh[1],
                     &ctx->Fv, &ctx->Fh};
  for (float **b : cubes) {
    if ((rc = dmalloc(ctx, (void **)b, np * sizeof(float)))) {
      free_all(ctx);
      return rc;
    }
  }
  if (is_ssst(ctx)) {
    float **ssst[] = {&ctx->Fs, &ctx->Zs[0], &ctx->Zs[1]};
    for (float **b : ssst) {
      if ((rc = dmalloc(ctx, (void **)b, np * sizeof(float)))) {
        free_all(ctx);
        return rc;
      }
    }
  }
  const int fb_cap = dm.P < kFbQueueMax ? (int)dm.P : kFbQueueMax;
  if ((rc = dmalloc(ctx, (void **)&ctx->Y, ny * sizeof(float))) ||
      (rc = dmalloc(ctx, (void **)&ctx->W, nw * sizeof(float))) ||
      (rc = dmalloc(ctx, (void **)&ctx->fb_list, (size_t)fb_cap * sizeof(int)))) {
    free_all(ctx);
    return rc;
  }
  ctx->fb_cap = fb_cap;
  ctx->cap_np = np;
  ctx->cap_y = ny;
  ctx->cap_w = nw;
  return S3TTV_OK;
}

Dims make_dims(int N1, int N2, int N3) {
  Dims dm;
  dm.N1 = N1;
  dm.N2 = N2;
  dm.N3 = N3;
  dm.N3p = round4(N3);
  dm.P = (long long)N1 * N2;
  dm.Np = dm.P * dm.N3p;
  return dm;
}

// The polish threshold of the block eigen-solves (S3TTV_OPT_JACOBI_POLISH_TOL):
// the option's value, at most the tolerance; by default 2.5e-7, near the FP32
// rounding of a row pair's dot product.  Every sweep rotates each pair above
// it; only a pair above the tolerance makes the solve run another sweep.  A
// last sweep whose rotations all stay below the tolerance tau changes a pair
// it already met by at most about n tau^2 (2.6e-6 at tau = 1e-4, n = 256), so
// the default tolerance 1e-4 leaves the per-operator errors as they were at
// tau = 2e-6 (measured on GB300 for k = 5..16) with one sweep fewer.
constexpr float kDefaultPolish = 2.5e-7f;
float jacobi_polish_for(const s3ttv_ctx *ctx) {
  const float tol = ctx->jacobi_tol;
  const float p = ctx->jacobi_polish > 0.f ? ctx->jacobi_polish : kDefaultPolish;
  return p < tol ? p : tol;
}

// Block-dual launch shape: one CTA per group of block_dual_group() blocks, a
// persistent grid of as many CTAs as fit on the device at once.  The kernel
// variant sized for the most CTAs per SM whose shared memory fits is taken.
struct BdShape {
  int rs = 0;       // shared-memory row stride (floats) of the block copies
  size_t smem = 0;  // dynamic shared memory per CTA
  int grid = 0;
  BdVariant v;
  bool large = false;  // block_dual_large.cu (k > 5)
  size_t fb_smem = 0;  // dynamic shared memory of the FP64 re-solve (0: not available)
  size_t rows_bytes = 0;  // global scratch of the large kernel's grid (ensure_rows)
};

// The large kernel's global scratch for shape sh.  Call it after
// ensure_problem_buffers, whose reallocation frees every buffer of the context.
int ensure_rows(s3ttv_ctx *ctx, const BdShape &sh) {
  if (sh.rows_bytes <= ctx->cap_rows) return S3TTV_OK;
  if (ctx->rows) {
    cudaFree(ctx->rows);
    ctx->bytes -= ctx->cap_rows;
    ctx->rows = nullptr;
    ctx->cap_rows = 0;
  }
  int rc = dmalloc(ctx, (void **)&ctx->rows, sh.rows_bytes);
  if (rc) return rc;
  ctx->cap_rows = sh.rows_bytes;
  return S3TTV_OK;
}

// The launch shape of one block-dual form of the k <= 5 kernel: tensor cores
// (tc) or CUDA cores, compiled for minb CTAs per SM.  Fails (S3TTV_EUNSUPPORTED)
// when that form is not compiled or does not fit.
int block_dual_variant_shape(s3ttv_ctx *ctx, const Dims &dm, int k, int tc, int minb, BdShape *sh) {
  sh->large = false;
  sh->v.k = k;
  sh->v.tc = tc;
  sh->v.minb = minb;
  if (!block_dual_has(sh->v)) return fail(ctx, S3TTV_EUNSUPPORTED, "form tc=%d minb=%d not compiled", tc, minb);
  sh->rs = block_dual_row_stride(dm.N3p);
  sh->smem = block_dual_smem_bytes(sh->v, dm.N3p);
  int dev_max = 0;
  cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  if (sh->smem == 0 || sh->smem > (size_t)dev_max) return fail(ctx, S3TTV_EUNSUPPORTED, "form does not fit");
  cudaError_t e = block_dual_prepare(sh->v, sh->smem);
  if (e != cudaSuccess) return fail(ctx, S3TTV_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
  int per_sm = 0;
  e = block_dual_occupancy(sh->v, sh->smem, &per_sm);
  if (e != cudaSuccess) return fail(ctx, S3TTV_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
  if (per_sm < 1) return fail(ctx, S3TTV_EUNSUPPORTED, "form does not fit on an SM");
  long long g = (long long)ctx->num_sms * per_sm;
  const long long groups = (dm.P + block_dual_group() - 1) / block_dual_group();
  if (g > groups) g = groups;
  sh->grid = (int)g;
  return S3TTV_OK;
}

int block_dual_shape(s3ttv_ctx *ctx, const Dims &dm, int k, BdShape *sh) {
  if (dm.P > 2147483647LL)  // the kernels index pixels with 32-bit integers
    return fail(ctx, S3TTV_EUNSUPPORTED, "N1 * N2 = %lld pixels: this library supports fewer than 2^31", dm.P);
  if (dm.Np / 4 > 2147483647LL)  // and float4 chunks of bands with 32-bit integers
    return fail(ctx, S3TTV_EUNSUPPORTED, "%lld voxels: this library supports fewer than 2^33", dm.Np);
  sh->v.k = k;
  sh->v.tc = ctx->tensor_cores;
  const bool stacked = ctx->layout == S3TTV_LAYOUT_STACKED;
  const int parts = row_parts(ctx);
  if (stacked && k > kMaxStackedK)
    return fail(ctx, S3TTV_EUNSUPPORTED, "k = %d: the stacked layout supports k <= %d", k, kMaxStackedK);
  if (parts == 3 && (stacked || ctx->open_s))
    return fail(ctx, S3TTV_EUNSUPPORTED, "SSST takes the paper layout and the periodic spectral boundary");
  {  // the FP64 re-solve of blocks whose FP32 eigen-solve reaches the sweep cap
    int dev_max = 0;
    cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    const size_t fs = fallback_smem_bytes(stacked ? 2 * k * k : k * k);
    sh->fb_smem = 0;
    if (fs <= (size_t)dev_max) {
      cudaError_t e = fallback_prepare(fs);
      if (e != cudaSuccess) return fail(ctx, S3TTV_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
      sh->fb_smem = fs;
    }
  }
  if (parts == 3 && k > kMaxStackedK)
    return fail(ctx, S3TTV_EUNSUPPORTED, "k = %d: SSST supports k <= %d", k, kMaxStackedK);
  if (stacked || parts == 3 || k >= kMinLargeK) {  // one CTA per block at a time; FP32 CUDA cores
    sh->large = true;
    sh->smem = block_dual_large_smem_bytes(k, stacked, parts);
    int dev_max = 0;
    cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
    if (sh->smem > (size_t)dev_max)
      return fail(ctx, S3TTV_EUNSUPPORTED, "a %dx%d block needs %zu bytes of shared memory (device limit %d)", k, k,
                  sh->smem, dev_max);
    cudaError_t e = block_dual_large_prepare(k, stacked, sh->smem, parts);
    if (e != cudaSuccess) return fail(ctx, S3TTV_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    int per_sm = 0;
    e = block_dual_large_occupancy(k, stacked, sh->smem, &per_sm, parts);
    if (e != cudaSuccess) return fail(ctx, S3TTV_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
    if (per_sm < 1) per_sm = 1;
    long long g = (long long)ctx->num_sms * per_sm;
    if (g > dm.P) g = dm.P;
    sh->grid = (int)g;
    // blocks above kMaxSmemRows rows: their two n x n matrices per CTA in global memory
    sh->rows_bytes = block_dual_large_rows_floats(k, stacked, parts) * sizeof(float) * (size_t)g;
    return S3TTV_OK;
  }
  sh->rs = block_dual_row_stride(dm.N3p);
  sh->smem = block_dual_smem_bytes(sh->v, dm.N3p);
  int dev_max = 0;
  cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device);
  if (dev_max <= 0) dev_max = 227 * 1024;
  if (sh->smem == 0 || sh->smem > (size_t)dev_max)
    return fail(ctx, S3TTV_EUNSUPPORTED, "a %dx%dx%d block needs %zu bytes of shared memory (device limit %d)", k, k,
                dm.N3, sh->smem, dev_max);
  if (ctx->tuned_tc >= 0 && ctx->tuned_k == k && ctx->tuned_n3p == dm.N3p) {
    // the autotuned form (block_dual_variant_shape checked it when it was chosen)
    return block_dual_variant_shape(ctx, dm, k, ctx->tuned_tc, ctx->tuned_minb, sh);
  }
  int per_sm = 0;
  for (int minb = 5; minb >= 4; --minb) {
    sh->v.minb = minb;
    if (!block_dual_has(sh->v)) continue;  // variant not compiled
    cudaError_t e = block_dual_prepare(sh->v, sh->smem);
    if (e != cudaSuccess) return fail(ctx, S3TTV_ECUDA, "cudaFuncSetAttribute: %s", cudaGetErrorString(e));
    e = block_dual_occupancy(sh->v, sh->smem, &per_sm);
    if (e != cudaSuccess) return fail(ctx, S3TTV_ECUDA, "occupancy query: %s", cudaGetErrorString(e));
    if (per_sm >= minb) break;
  }
  if (per_sm < 1) per_sm = 1;
  long long g = (long long)ctx->num_sms * per_sm;
  const long long groups = (dm.P + block_dual_group() - 1) / block_dual_group();
  if (g > groups) g = groups;
  sh->grid = (int)g;
  return S3TTV_OK;
}

int check_problem(s3ttv_ctx *ctx, const float *v, int N1, int N2, int N3, float eps, float alpha, float beta,
                  float mu_min, float mu_max, int k) {
  if (!ctx) return S3TTV_EINVAL;
  if (!v) return fail(ctx, S3TTV_EINVAL, "v is NULL");
  if (k < 1) return fail(ctx, S3TTV_EINVAL, "k = %d must be >= 1", k);
  if (N1 < k || N2 < k) return fail(ctx, S3TTV_EINVAL, "N1 = %d and N2 = %d must be >= k = %d", N1, N2, k);
  if (N3 < 2) return fail(ctx, S3TTV_EINVAL, "N3 = %d must be >= 2", N3);
  if (!(std::isfinite(eps) && eps >= 0.f)) return fail(ctx, S3TTV_EINVAL, "eps must be finite and >= 0");
  if (!(std::isfinite(alpha) && alpha >= 0.f)) return fail(ctx, S3TTV_EINVAL, "alpha must be finite and >= 0");
  if (!(std::isfinite(beta) && beta >= 0.f)) return fail(ctx, S3TTV_EINVAL, "beta must be finite and >= 0");
  if (!(std::isfinite(mu_min) && std::isfinite(mu_max) && mu_min < mu_max))
    return fail(ctx, S3TTV_EINVAL, "need finite mu_min < mu_max");
  if ((long long)N1 * N2 * (long long)N3 > (1ll << 40)) return fail(ctx, S3TTV_EINVAL, "cube too large");
  if (k > kMaxK) return fail(ctx, S3TTV_EUNSUPPORTED, "k = %d: this library supports k <= %d", k, kMaxK);
  return S3TTV_OK;
}

// Step sizes (u, s, t, Y, y2, y3).  S3TTV: eq. (stepsize_denoising) under the
// policy; STV and SSTV: the exact Lemma 1 values of their operators (column
// abs-sums 4k^2 and 8 of P_l D and D D_s, row abs-sums 2 and 4, plus the
// identity of y3).
void step_sizes(int N1, int N2, int k, int policy, double g[6], int reg = S3TTV_REG_S3TTV, double omega = 0.05) {
  const double L = (double)N1 * (double)N2;
  g[0] = policy == S3TTV_STEP_PC_EXACT ? 1.0 / (8.0 * k * k + 1.0) : 1.0 / (8.0 * L + 1.0);
  g[1] = 1.0;
  g[2] = 1.0 / 3.0;
  g[3] = 0.25;
  g[4] = 0.5;
  g[5] = 1.0 / 3.0;
  if (reg == S3TTV_REG_STV) {
    g[0] = 1.0 / (4.0 * k * k + 1.0);
    g[3] = 0.5;
  } else if (reg == S3TTV_REG_SSTV) {
    g[0] = 1.0 / 9.0;
  } else if (reg == S3TTV_REG_HSSTV1 || reg == S3TTV_REG_HSSTV2) {
    g[0] = 1.0 / (9.0 + 4.0 * omega);  // gamma_Y = 1/4 serves all four dual parts (omega <= 2)
  } else if (reg == S3TTV_REG_SSST) {
    g[0] = 1.0 / (6.0 * k * k + 1.0);  // column abs-sum 6k^2 of P_l [D_v; D_h; D_s], plus y3's 1
    g[3] = 0.5;                          // row abs-sum 2 of a first-order difference
  }
}

// Copy a caller cube (host or device, [N1][N2][N3]) into an internal padded cube.
int load_cube(s3ttv_ctx *ctx, const float *src, float *dst, float scale) {
  const Dims &dm = ctx->dm;
  const float *from = src;
  if (!is_device_ptr(src)) {
    int rc = ensure_stage(ctx, (size_t)dm.P * dm.N3);
    if (rc) return rc;
    CU(cudaMemcpyAsync(ctx->stage, src, sizeof(float) * dm.P * dm.N3, cudaMemcpyHostToDevice, ctx->stream));
    from = ctx->stage;
  }
  CU(launch_pad_cube(from, dst, dm, scale, ctx->stream));
  return S3TTV_OK;
}

int store_cube(s3ttv_ctx *ctx, const float *src, float *dst, const double *scale_dev) {
  const Dims &dm = ctx->dm;
  if (is_device_ptr(dst)) {
    CU(launch_unpad_cube(src, dst, dm, scale_dev, ctx->stream));
    return S3TTV_OK;
  }
  int rc = ensure_stage(ctx, (size_t)dm.P * dm.N3);
  if (rc) return rc;
  CU(launch_unpad_cube(src, ctx->stage, dm, scale_dev, ctx->stream));
  CU(cudaMemcpyAsync(dst, ctx->stage, sizeof(float) * dm.P * dm.N3, cudaMemcpyDeviceToHost, ctx->stream));
  return S3TTV_OK;
}

int load_Y(s3ttv_ctx *ctx, const float *src) {
  const Dims &dm = ctx->dm;
  const int ncubes = ctx->reg == S3TTV_REG_SSTV ? 2 : (is_hsstv(ctx) ? 4 : 0);
  if (ncubes) {  // SSTV (Yv, Yh) / HSSTV (four parts): cubes
    int rc = S3TTV_OK;
    for (int m = 0; m < ncubes && !rc; ++m) rc = load_cube(ctx, src + m * dm.P * dm.N3, ctx->Y + m * dm.Np, 1.f);
    return rc;
  }
  const size_t ne = (size_t)dm.P * ctx->k * ctx->k * row_parts(ctx) * dm.N3;
  const float *from = src;
  if (!is_device_ptr(src)) {
    int rc = ensure_stage(ctx, ne);
    if (rc) return rc;
    CU(cudaMemcpyAsync(ctx->stage, src, sizeof(float) * ne, cudaMemcpyHostToDevice, ctx->stream));
    from = ctx->stage;
  }
  CU(launch_Y_to_internal(from, ctx->Y, dm, ctx->k, ctx->stream, ctx->layout == S3TTV_LAYOUT_STACKED,
                          row_parts(ctx)));
  return S3TTV_OK;
}

int store_Y(s3ttv_ctx *ctx, float *dst) {
  const Dims &dm = ctx->dm;
  const int ncubes = ctx->reg == S3TTV_REG_SSTV ? 2 : (is_hsstv(ctx) ? 4 : 0);
  if (ncubes) {
    int rc = S3TTV_OK;
    for (int m = 0; m < ncubes && !rc; ++m) rc = store_cube(ctx, ctx->Y + m * dm.Np, dst + m * dm.P * dm.N3, nullptr);
    return rc;
  }
  const size_t ne = (size_t)dm.P * ctx->k * ctx->k * row_parts(ctx) * dm.N3;
  if (is_device_ptr(dst)) {
    CU(launch_Y_to_external(ctx->Y, dst, dm, ctx->k, ctx->stream, ctx->layout == S3TTV_LAYOUT_STACKED,
                            row_parts(ctx)));
    return S3TTV_OK;
  }
  int rc = ensure_stage(ctx, ne);
  if (rc) return rc;
  CU(launch_Y_to_external(ctx->Y, ctx->stage, dm, ctx->k, ctx->stream, ctx->layout == S3TTV_LAYOUT_STACKED,
                          row_parts(ctx)));
  CU(cudaMemcpyAsync(dst, ctx->stage, sizeof(float) * ne, cudaMemcpyDeviceToHost, ctx->stream));
  return S3TTV_OK;
}

__global__ void begin_iterate_kernel(Scalars *sc, int n, float tol) {
  sc->iter_limit = sc->iter + n;
  sc->done = 0;
  sc->status = 0;
  sc->tol = tol;
  sc->jacobi_fail = 0u;
  sc->jacobi_sweeps = 0ull;
  sc->fb_total = 0u;
  sc->fo_blocks = 0ull;
}

__global__ void set_c3_kernel(Scalars *sc, double c3) { sc->c3 = c3; }

// One pass of Alg. 1, enqueued on the context stream.  `par` selects the current
// t / Z buffers; the pass writes the other ones.
// The block-dual arguments of one pass at parity par.
BlockDualArgs make_bd_args(s3ttv_ctx *ctx, int par, const BdShape &bd) {
  BlockDualArgs ba;
  ba.Y = ctx->Y;
  ba.Fv = ctx->Fv;
  ba.Fh = ctx->Fh;
  ba.Fs = ctx->Fs;
  ba.Zv = ctx->Zv[par ^ 1];
  ba.Zh = ctx->Zh[par ^ 1];
  ba.Zs = ctx->Zs[par ^ 1];
  ba.dm = ctx->dm;
  ba.gY = (float)ctx->gam[3];
  ba.rs = bd.rs;
  ba.max_sweeps = ctx->jacobi_max_sweeps;
  ba.tol = ctx->jacobi_tol;
  ba.polish = jacobi_polish_for(ctx);
  ba.fo_tol = bd.large ? 0.f : ctx->first_order;
  ba.sc = ctx->sc;
  ba.W = ctx->warm_start ? ctx->W : nullptr;
  ba.w_stride = ctx->w_stride;
  ba.warm = ctx->warm_start && ctx->warm_valid;
  const bool fb = ctx->fp64_fallback && bd.fb_smem > 0;
  ba.fb_list = fb ? ctx->fb_list : nullptr;
  ba.fb_cap = fb ? ctx->fb_cap : 0;
  ba.rows = ctx->rows;
  ba.rows_cap = ctx->cap_rows / sizeof(float);
  return ba;
}

// One pass of Alg. 1 (part 0), or its steps before the block duals (part 1:
// primal step, l1-ball thresholds, D D_s ubar) or after them (part 2: the FP64
// re-solve queue, the dual step, finalize); the batched solve launches the
// block duals of all its problems in between.
int enqueue_pass(s3ttv_ctx *ctx, int par, int grid_e, const BdShape &bd,
                 cudaEvent_t *ev, int part = 0) {
  const Dims &dm = ctx->dm;
  cudaStream_t st = ctx->stream;
  NvtxPhase ph(ctx->nvtx);
  if (part == 2) {
    const BlockDualArgs ba = make_bd_args(ctx, par, bd);
    if (ba.fb_list) {
      CU(launch_fallback(ba, ctx->k, ctx->layout == S3TTV_LAYOUT_STACKED, row_parts(ctx), ctx->num_sms,
                         bd.fb_smem, st));
      ctx->launches += 1;
    }
    if (ctx->warm_start) ctx->warm_valid = true;
  }
  if (part != 2) {
  ph.next("primal (steps 2-7)");
  if (ev) CU(cudaEventRecord(ev[0], st));
  PrimalArgs pa;
  pa.Zv = ctx->Zv[par];
  pa.Zh = ctx->Zh[par];
  pa.Znv = ctx->Zv[par ^ 1];
  pa.Znh = ctx->Zh[par ^ 1];
  pa.u = ctx->u;
  pa.ubar = ctx->ubar;
  pa.s = ctx->s;
  pa.t = ctx->t[par];
  pa.y2 = ctx->y2;
  pa.d = ctx->d;
  pa.zs = ctx->zs;
  pa.zt = ctx->zt;
  pa.dm = dm;
  pa.gu = (float)ctx->gam[0];
  pa.gs = (float)ctx->gam[1];
  pa.gt = (float)ctx->gam[2];
  pa.lo = ctx->mu_min;
  pa.hi = ctx->mu_max;
  pa.sc = ctx->sc;
  pa.part = ctx->part;
  pa.hcnt = ctx->hcnt;
  pa.hsum = ctx->hsum;
  pa.no_ds = ctx->reg == S3TTV_REG_STV || is_ssst(ctx);
  if (is_ssst(ctx)) {
    pa.Zs = ctx->Zs[par];
    pa.Zns = ctx->Zs[par ^ 1];
  }
  if (is_hsstv(ctx)) {
    pa.Z1v = ctx->Y + 2 * dm.Np;
    pa.Z1h = ctx->Y + 3 * dm.Np;
    pa.w1 = ctx->hsstv_omega;
  }
  CU(launch_primal(pa, grid_e, st));
  if (ev) CU(cudaEventRecord(ev[1], st));
  ph.next("l1-ball thresholds (steps 3-4)");

  L1Args la;
  la.x[0] = ctx->zs;
  la.x[1] = ctx->zt;
  la.n = dm.Np;
  la.nprob = 2;
  la.sc = ctx->sc;
  la.hcnt = ctx->hcnt;
  la.hsum = ctx->hsum;
  CU(launch_l1_scan(la, 1, st));
  CU(launch_l1_hist(la, 2, grid_e, st));
  CU(launch_l1_scan(la, 2, st));
  CU(launch_l1_hist(la, 3, grid_e, st));
  CU(launch_l1_scan(la, 3, st));
  if (ev) CU(cudaEventRecord(ev[2], st));

  ph.next("block dual (steps 8-11)");
  if (ctx->reg == S3TTV_REG_SSTV) {
    CU(launch_sstv_dual(ctx->ubar, ctx->Y, ctx->Y + dm.Np, ctx->Zv[par ^ 1], ctx->Zh[par ^ 1], dm,
                        (float)ctx->gam[3], grid_e, st));
  } else if (is_hsstv(ctx)) {
    CU(launch_hsstv_dual(ctx->ubar, ctx->Y, ctx->Zv[par ^ 1], ctx->Zh[par ^ 1], dm, (float)ctx->gam[3],
                         ctx->hsstv_omega, ctx->reg == S3TTV_REG_HSSTV2, grid_e, st));
  } else {
  CU(launch_xfield(ctx->ubar, ctx->Fv, ctx->Fh, dm, grid_e, st, ctx->open_s,
                   ctx->reg == S3TTV_REG_STV || is_ssst(ctx), ctx->Fs));
  if (part == 1) {
    ctx->launches += 7;  // primal, three scans, two histograms, xfield
    return S3TTV_OK;
  }
  const BlockDualArgs ba = make_bd_args(ctx, par, bd);
  const bool fb = ba.fb_list != nullptr;
  if (bd.large)
    CU(launch_block_dual_large(ba, ctx->k, ctx->layout == S3TTV_LAYOUT_STACKED, bd.grid, bd.smem, st,
                               row_parts(ctx)));
  else CU(launch_block_dual(ba, bd.v, bd.grid, bd.smem, st));
  if (fb) {
    CU(launch_fallback(ba, ctx->k, ctx->layout == S3TTV_LAYOUT_STACKED, row_parts(ctx), ctx->num_sms, bd.fb_smem,
                       st));
    ctx->launches += 1;
  }
  if (ctx->warm_start) ctx->warm_valid = true;
  }
  if (ev) CU(cudaEventRecord(ev[3], st));
  }  // part != 2

  ph.next("dual (steps 12-13)");
  DualArgs da;
  da.zs = ctx->zs;
  da.zt = ctx->zt;
  da.s_old = ctx->s;
  da.t_old = ctx->t[par];
  da.ubar = ctx->ubar;
  da.v = ctx->v;
  da.s_new = ctx->s;
  da.t_new = ctx->t[par ^ 1];
  da.y2 = ctx->y2;
  da.d = ctx->d;
  da.dm = dm;
  da.g2 = (float)ctx->gam[4];
  da.g3 = (float)ctx->gam[5];
  da.sc = ctx->sc;
  da.part = ctx->part + 2 * grid_e;
  CU(launch_dual(da, grid_e, st));
  if (ev) CU(cudaEventRecord(ev[4], st));

  FinalizeArgs fa;
  fa.sc = ctx->sc;
  fa.part_primal = ctx->part;
  fa.grid_p = grid_e;
  fa.part_dual = ctx->part + 2 * grid_e;
  fa.grid_d = grid_e;
  fa.eps = ctx->eps;
  fa.g3 = ctx->gam[5];
  ph.next("finalize (step 14, stop rule)");
  CU(launch_finalize(fa, st));
  if (ev) CU(cudaEventRecord(ev[5], st));
  if (part == 2) {
    ctx->launches += 2;  // dual, finalize (the block duals are counted by the batch)
    return S3TTV_OK;
  }
  // SSTV and HSSTV: one elementwise dual kernel in place of xfield + block dual
  ctx->launches += (ctx->reg == S3TTV_REG_SSTV || is_hsstv(ctx)) ? kLaunchesPerPass - 1 : kLaunchesPerPass;
  return S3TTV_OK;
}

double now_s() {
  return std::chrono::duration<double>(std::chrono::steady_clock::now().time_since_epoch()).count();
}

constexpr int kEvPerPass = S3TTV_KERNEL_CLASSES + 1;  // boundaries around the five classes

void destroy_events(s3ttv_ctx *c) {
  for (int i = 0; i < kEvPerPass * c->ev_passes; ++i) cudaEventDestroy(c->ev[i]);
  delete[] c->ev;
  c->ev = nullptr;
  c->ev_passes = 0;
}

int ensure_events(s3ttv_ctx *ctx, int passes) {
  if (passes <= ctx->ev_passes) return S3TTV_OK;
  destroy_events(ctx);
  ctx->ev = new (std::nothrow) cudaEvent_t[(size_t)kEvPerPass * passes];
  if (!ctx->ev) return fail(ctx, S3TTV_ENOMEM, "event pool");
  for (int i = 0; i < kEvPerPass * passes; ++i) {
    cudaError_t e = cudaEventCreate(&ctx->ev[i]);
    if (e != cudaSuccess) {
      for (int j = 0; j < i; ++j) cudaEventDestroy(ctx->ev[j]);
      delete[] ctx->ev;
      ctx->ev = nullptr;
      return fail(ctx, S3TTV_ECUDA, "cudaEventCreate: %s", cudaGetErrorString(e));
    }
  }
  ctx->ev_passes = passes;
  return S3TTV_OK;
}

// Add the elapsed times of `passes` recorded passes to the per-class totals.
int collect_events(s3ttv_ctx *ctx, int passes) {
  for (int p = 0; p < passes; ++p) {
    cudaEvent_t *e = ctx->ev + (size_t)kEvPerPass * p;
    for (int c = 0; c < S3TTV_KERNEL_CLASSES; ++c) {
      float ms = 0.f;
      CU(cudaEventElapsedTime(&ms, e[c], e[c + 1]));
      ctx->prof_ms[c] += ms;
      ctx->prof_n[c] += c == S3TTV_KERNEL_L1_SEARCH ? 5 : 1;
    }
  }
  return S3TTV_OK;
}

}  // namespace

extern "C" {

const char *s3ttv_strerror(int status) {
  switch (status) {
    case S3TTV_OK: return "ok (stop rule fired)";
    case S3TTV_MAXITER: return "iteration cap reached";
    case S3TTV_EINVAL: return "invalid argument";
    case S3TTV_ENOMEM: return "device allocation failed";
    case S3TTV_ECUDA: return "CUDA runtime error";
    case S3TTV_ENUMERIC: return "NaN or Inf in the iterates";
    case S3TTV_EUNSUPPORTED: return "not supported by this library";
    case S3TTV_ESTATE: return "no problem set up";
    case S3TTV_ETOOBIG: return "input larger than the allocation-free entry point takes";
    default: return "unknown status";
  }
}

const char *s3ttv_last_error(const s3ttv_ctx *ctx) { return ctx ? ctx->err : "null context"; }

long long s3ttv_workspace_bytes(const s3ttv_ctx *ctx) { return ctx ? (long long)ctx->bytes : 0; }

long long s3ttv_launch_count(const s3ttv_ctx *ctx) {
  if (!ctx) return 0;
  long long n = ctx->launches;
  for (const s3ttv_ctx *m : ctx->members) n += m->launches;  // batched solves
  return n;
}

int s3ttv_kernel_stats(const s3ttv_ctx *ctx, double *ms, long long *launches) {
  if (!ctx) return S3TTV_EINVAL;
  for (int c = 0; c < S3TTV_KERNEL_CLASSES; ++c) {
    if (ms) ms[c] = ctx->prof_ms[c];
    if (launches) launches[c] = ctx->prof_n[c];
  }
  return S3TTV_OK;
}

int s3ttv_create(s3ttv_ctx **out, int device, void *stream) {
  if (!out) return S3TTV_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return S3TTV_ECUDA;
  }
  if (device < 0 || device >= ndev) return S3TTV_EINVAL;
  s3ttv_ctx *ctx = new (std::nothrow) s3ttv_ctx();
  if (!ctx) return S3TTV_ENOMEM;
  ctx->device = device;
  DeviceGuard g(device);
  cudaDeviceGetAttribute(&ctx->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (ctx->num_sms <= 0) ctx->num_sms = 1;
  if (stream) {
    ctx->stream = (cudaStream_t)stream;
  } else {
    if (cudaStreamCreateWithFlags(&ctx->stream, cudaStreamNonBlocking) != cudaSuccess) {
      cudaGetLastError();
      delete ctx;
      return S3TTV_ECUDA;
    }
    ctx->own_stream = true;
  }
  *out = ctx;
  return S3TTV_OK;
}

void s3ttv_destroy(s3ttv_ctx *ctx) {
  if (!ctx) return;
  for (s3ttv_ctx *m : ctx->members) s3ttv_destroy(m);
  ctx->members.clear();
  {
    DeviceGuard g(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    free_all(ctx);
    destroy_events(ctx);
    if (ctx->own_stream) cudaStreamDestroy(ctx->stream);
  }
  delete ctx;
}

int s3ttv_set_option(s3ttv_ctx *ctx, int key, double value) {
  if (!ctx) return S3TTV_EINVAL;
  switch (key) {
    case S3TTV_OPT_STEP_POLICY:
      if (value != S3TTV_STEP_PAPER && value != S3TTV_STEP_PC_EXACT)
        return fail(ctx, S3TTV_EINVAL, "unknown step policy %g", value);
      ctx->step_policy = (int)value;
      if (ctx->ready) step_sizes(ctx->dm.N1, ctx->dm.N2, ctx->k, ctx->step_policy, ctx->gam, ctx->reg, ctx->hsstv_omega);
      return S3TTV_OK;
    case S3TTV_OPT_CHECK_EVERY:
      if (!(value >= 1 && value <= 1e6)) return fail(ctx, S3TTV_EINVAL, "check_every must be in [1, 1e6]");
      ctx->check_every = (int)value;
      return S3TTV_OK;
    case S3TTV_OPT_JACOBI_MAX_SWEEPS:
      if (!(value >= 1 && value <= 64)) return fail(ctx, S3TTV_EINVAL, "jacobi sweeps must be in [1, 64]");
      ctx->jacobi_max_sweeps = (int)value;
      return S3TTV_OK;
    case S3TTV_OPT_JACOBI_TOL:
      if (!(value > 0 && value < 1)) return fail(ctx, S3TTV_EINVAL, "jacobi tol must be in (0, 1)");
      ctx->jacobi_tol = (float)value;
      return S3TTV_OK;
    case S3TTV_OPT_FIRST_ORDER:
      if (!(value >= 0 && value < 1)) return fail(ctx, S3TTV_EINVAL, "first-order bound must be in [0, 1)");
      ctx->first_order = (float)value;
      return S3TTV_OK;
    case S3TTV_OPT_BATCH_WORKLIST:
      if (value != 0 && value != 1) return fail(ctx, S3TTV_EINVAL, "batch_worklist must be 0 or 1");
      ctx->batch_worklist = (int)value;
      return S3TTV_OK;
    case S3TTV_OPT_JACOBI_POLISH_TOL:
      if (!(value >= 0 && value < 1)) return fail(ctx, S3TTV_EINVAL, "jacobi polish tolerance must be in [0, 1)");
      ctx->jacobi_polish = (float)value;
      return S3TTV_OK;
    case S3TTV_OPT_TENSOR_CORES:
      ctx->tuned_tc = -1;
      if (value != 0 && value != 1 && value != 2) return fail(ctx, S3TTV_EINVAL, "tensor_cores must be 0, 1 or 2");
      ctx->tensor_cores = (int)value;
      return S3TTV_OK;
    case S3TTV_OPT_WARM_START:
      if (value != 0 && value != 1) return fail(ctx, S3TTV_EINVAL, "warm_start must be 0 or 1");
      ctx->warm_start = value == 1;
      ctx->warm_valid = false;
      return S3TTV_OK;
    case S3TTV_OPT_LAYOUT:
      if (value != S3TTV_LAYOUT_PAPER && value != S3TTV_LAYOUT_STACKED)
        return fail(ctx, S3TTV_EINVAL, "layout must be S3TTV_LAYOUT_PAPER or S3TTV_LAYOUT_STACKED");
      if ((int)value != ctx->layout) {
        ctx->layout = (int)value;
        ctx->ready = false;  // the block duals change meaning: set the problem up again
        ctx->warm_valid = false;
      }
      return S3TTV_OK;
    case S3TTV_OPT_SPECTRAL_BOUNDARY:
      if (value != S3TTV_SPECTRAL_PERIODIC && value != S3TTV_SPECTRAL_OPEN)
        return fail(ctx, S3TTV_EINVAL, "spectral boundary must be S3TTV_SPECTRAL_PERIODIC or S3TTV_SPECTRAL_OPEN");
      if ((int)value != ctx->open_s) {
        ctx->open_s = (int)value;
        ctx->ready = false;
        ctx->warm_valid = false;
      }
      return S3TTV_OK;
    case S3TTV_OPT_ALLOC_LIMIT:
      if (!(value >= 0.0 && value < 1.8e19)) return fail(ctx, S3TTV_EINVAL, "alloc_limit must be >= 0 bytes");
      ctx->alloc_limit = (size_t)value;
      return S3TTV_OK;
    case S3TTV_OPT_NVTX:
      if (value != 0 && value != 1) return fail(ctx, S3TTV_EINVAL, "nvtx must be 0 or 1");
      ctx->nvtx = value == 1;
      return S3TTV_OK;
    case S3TTV_OPT_FP64_FALLBACK:
      if (value != 0 && value != 1) return fail(ctx, S3TTV_EINVAL, "fp64_fallback must be 0 or 1");
      ctx->fp64_fallback = value == 1;
      return S3TTV_OK;
    case S3TTV_OPT_HSSTV_OMEGA:
      if (!(value > 0.0 && value <= 2.0)) return fail(ctx, S3TTV_EINVAL, "HSSTV omega must be in (0, 2]");
      ctx->hsstv_omega = (float)value;
      if (ctx->ready) step_sizes(ctx->dm.N1, ctx->dm.N2, ctx->k, ctx->step_policy, ctx->gam, ctx->reg, ctx->hsstv_omega);
      return S3TTV_OK;
    case S3TTV_OPT_AUTOTUNE:
      if (value != 0 && value != 1) return fail(ctx, S3TTV_EINVAL, "autotune must be 0 or 1");
      ctx->autotune = (int)value;
      ctx->tuned_tc = -1;  // choose again on the next passes
      return S3TTV_OK;
    case S3TTV_OPT_REGULARIZER:
      if (!(value == S3TTV_REG_S3TTV || value == S3TTV_REG_STV || value == S3TTV_REG_SSTV ||
            value == S3TTV_REG_HSSTV1 || value == S3TTV_REG_HSSTV2 || value == S3TTV_REG_SSST))
        return fail(ctx, S3TTV_EINVAL, "unknown regularizer %g", value);
      if ((int)value != ctx->reg) {
        ctx->reg = (int)value;
        ctx->ready = false;  // the duals change meaning: set the problem up again
        ctx->warm_valid = false;
      }
      return S3TTV_OK;
    case S3TTV_OPT_PROFILE:
      if (value != 0 && value != 1) return fail(ctx, S3TTV_EINVAL, "profile must be 0 or 1");
      ctx->profile = value == 1;
      for (int c = 0; c < S3TTV_KERNEL_CLASSES; ++c) {
        ctx->prof_ms[c] = 0.0;
        ctx->prof_n[c] = 0;
      }
      return S3TTV_OK;
    default:
      return fail(ctx, S3TTV_EINVAL, "unknown option key %d", key);
  }
}

int s3ttv_radii(long long N, double sigma, double p_s, double p_t, double rho, double *eps, double *alpha,
                double *beta) {
  if (!eps || !alpha || !beta || N < 1 || !(sigma >= 0) || !(p_s >= 0 && p_s <= 1) || !(p_t >= 0 && p_t <= 1) ||
      !(rho > 0))
    return S3TTV_EINVAL;
  *alpha = rho * (double)N * p_s / 2.0;
  *beta = rho * 0.5 * (double)N * p_t * (1.0 - p_s) / 2.0;
  *eps = sigma > 0 ? rho * std::sqrt(sigma * sigma * (double)N * (1.0 - p_s)) : 0.01;
  return S3TTV_OK;
}

int s3ttv_step_sizes(int N1, int N2, int k, int policy, double gammas[6]) {
  if (!gammas || N1 < 1 || N2 < 1 || k < 1) return S3TTV_EINVAL;
  if (policy != S3TTV_STEP_PAPER && policy != S3TTV_STEP_PC_EXACT) return S3TTV_EINVAL;
  step_sizes(N1, N2, k, policy, gammas);
  return S3TTV_OK;
}

int s3ttv_setup(s3ttv_ctx *ctx, const float *v, int N1, int N2, int N3, float eps, float alpha, float beta,
                float mu_min, float mu_max, int k) {
  int rc = check_problem(ctx, v, N1, N2, N3, eps, alpha, beta, mu_min, mu_max, k);
  if (rc) return rc;
  NvtxRange nr(ctx->nvtx, "s3ttv_setup");
  DeviceGuard g(ctx->device);
  ctx->ready = false;
  const Dims dm = make_dims(N1, N2, N3);
  BdShape bd;
  if ((rc = block_dual_shape(ctx, dm, k, &bd))) return rc;
  if ((rc = ensure_problem_buffers(ctx, dm, k))) return rc;
  ctx->dm = dm;
  ctx->k = k;
  ctx->eps = eps;
  ctx->alpha = alpha;
  ctx->beta = beta;
  ctx->mu_min = mu_min;
  ctx->mu_max = mu_max;
  step_sizes(N1, N2, k, ctx->step_policy, ctx->gam, ctx->reg, ctx->hsstv_omega);
  const size_t cb = sizeof(float) * dm.Np;
  if ((rc = load_cube(ctx, v, ctx->v, 1.f))) return rc;
  CU(cudaMemcpyAsync(ctx->u, ctx->v, cb, cudaMemcpyDeviceToDevice, ctx->stream));  // u0 = v
  float *zero[] = {ctx->s, ctx->t[0], ctx->t[1], ctx->y2, ctx->d, ctx->ubar, ctx->zs, ctx->zt,
                   ctx->Zv[0], ctx->Zv[1], ctx->Zh[0], ctx->Zh[1]};
  for (float *z : zero) CU(cudaMemsetAsync(z, 0, cb, ctx->stream));
  if (is_ssst(ctx))
    for (float *z : {ctx->Zs[0], ctx->Zs[1]}) CU(cudaMemsetAsync(z, 0, cb, ctx->stream));
  CU(cudaMemsetAsync(ctx->Y, 0, sizeof(float) * dm.P * k * k * row_parts(ctx) * dm.N3p, ctx->stream));
  CU(cudaMemsetAsync(ctx->hcnt, 0, sizeof(unsigned) * 2 * kHistBins, ctx->stream));
  CU(cudaMemsetAsync(ctx->hsum, 0, sizeof(double) * 2 * kHistBins, ctx->stream));
  CU(launch_init_scalars(ctx->sc, alpha, beta, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  ctx->parity = 0;
  ctx->warm_valid = false;
  ctx->ready = true;
  return S3TTV_OK;
}

int s3ttv_iterate(s3ttv_ctx *ctx, int n, float tol, s3ttv_info *info) {
  if (!ctx) return S3TTV_EINVAL;
  NvtxRange nr(ctx->nvtx, "s3ttv_iterate");
  const double t0 = now_s();
  if (info) memset(info, 0, sizeof(*info));
  if (!ctx->ready) return fail(ctx, S3TTV_ESTATE, "s3ttv_iterate before s3ttv_setup");
  if (n < 1) return fail(ctx, S3TTV_EINVAL, "n = %d must be >= 1", n);
  if (!(tol >= 0.f) || !std::isfinite(tol)) return fail(ctx, S3TTV_EINVAL, "tol must be finite and >= 0");
  DeviceGuard g(ctx->device);
  BdShape bd;
  int rc = block_dual_shape(ctx, ctx->dm, ctx->k, &bd);
  if (!rc) rc = ensure_rows(ctx, bd);
  if (rc) return rc;
  const int grid_e = elementwise_grid(ctx, ctx->dm.Np);
  Scalars hs;
  CU(cudaMemcpyAsync(&hs, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  const int iter0 = hs.iter;
  const int par0 = ctx->parity;
  begin_iterate_kernel<<<1, 1, 0, ctx->stream>>>(ctx->sc, n, tol);
  CU(cudaGetLastError());
  ctx->launches += 1;
  int enq = 0, par = par0;
  if (ctx->autotune && ctx->reg != S3TTV_REG_SSTV && !is_hsstv(ctx) && !bd.large &&
      !(ctx->tuned_tc >= 0 && ctx->tuned_k == ctx->k && ctx->tuned_n3p == ctx->dm.N3p)) {
    // Autotuning of the block-dual form: after two passes (the cold eigen-
    // solves), time one pass of every compiled form that fits, twice each, with
    // CUDA events, and keep the fastest.  Every timed pass is a pass of the solve.
    struct Cand { int tc, minb; BdShape sh; float ms = 1e30f; };
    std::vector<Cand> cands;
    for (int tc = 2; tc >= 0; --tc)
      for (int minb = 5; minb >= 4; --minb) {
        Cand c;
        c.tc = tc;
        c.minb = minb;
        c.sh.fb_smem = bd.fb_smem;  // the FP64 re-solve stays on while the forms are timed
        if (block_dual_variant_shape(ctx, ctx->dm, ctx->k, tc, minb, &c.sh) == S3TTV_OK) cands.push_back(c);
      }
    ctx->err[0] = 0;
    const int need = 2 + 2 * (int)cands.size();
    if (cands.size() > 1 && n >= need) {
      for (int w = 0; w < 2; ++w, ++enq, par ^= 1)
        if ((rc = enqueue_pass(ctx, par, grid_e, cands[0].sh, nullptr))) return rc;
      if ((rc = ensure_events(ctx, 1))) return rc;
      for (int rep = 0; rep < 2; ++rep)
        for (Cand &c : cands) {
          CU(cudaEventRecord(ctx->ev[0], ctx->stream));
          if ((rc = enqueue_pass(ctx, par, grid_e, c.sh, nullptr))) return rc;
          CU(cudaEventRecord(ctx->ev[1], ctx->stream));
          CU(cudaEventSynchronize(ctx->ev[1]));
          float ms = 0.f;
          CU(cudaEventElapsedTime(&ms, ctx->ev[0], ctx->ev[1]));
          if (ms < c.ms) c.ms = ms;
          ++enq;
          par ^= 1;
        }
      const Cand *best = &cands[0];
      for (const Cand &c : cands)
        if (c.ms < best->ms) best = &c;
      ctx->tuned_tc = best->tc;
      ctx->tuned_minb = best->minb;
      ctx->tuned_k = ctx->k;
      ctx->tuned_n3p = ctx->dm.N3p;
      ctx->tensor_cores = best->tc;
      bd = best->sh;
    }
  }
  while (enq < n) {
    const int chunk = n - enq < ctx->check_every ? n - enq : ctx->check_every;
    if (ctx->profile && (rc = ensure_events(ctx, chunk))) return rc;
    for (int c = 0; c < chunk; ++c) {
      cudaEvent_t *ev = ctx->profile ? ctx->ev + (size_t)kEvPerPass * c : nullptr;
      if ((rc = enqueue_pass(ctx, par, grid_e, bd, ev))) return rc;
      par ^= 1;
    }
    enq += chunk;
    CU(cudaMemcpyAsync(&hs, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
    CU(cudaStreamSynchronize(ctx->stream));
    if (ctx->profile) {
      // passes skipped after the stop flag are empty launches; count what ran
      const int ran = hs.iter - iter0 - (enq - chunk);
      if ((rc = collect_events(ctx, ran < chunk ? (ran > 0 ? ran : 0) : chunk))) return rc;
    }
    if (hs.done) break;
  }
  const int done_iters = hs.iter - iter0;
  ctx->parity = (par0 + done_iters) & 1;
  int status;
  if (hs.status == -4) {
    status = fail(ctx, S3TTV_ENUMERIC, "NaN or Inf after %d passes", done_iters);
  } else {
    status = hs.status == 1 ? S3TTV_OK : S3TTV_MAXITER;
  }
  if (info) {
    info->status = status;
    info->iters = done_iters;
    info->converged = hs.status == 1;
    info->jacobi_nonconverged = (int)hs.jacobi_fail;
    info->jacobi_fallbacks = (int)hs.fb_total;
    info->rel_change = hs.rel;
    info->seconds = now_s() - t0;
    info->jacobi_sweeps = done_iters > 0 ? (double)hs.jacobi_sweeps / ((double)done_iters * ctx->dm.P) : 0.0;
    info->first_order = done_iters > 0 ? (double)hs.fo_blocks / ((double)done_iters * ctx->dm.P) : 0.0;
  }
  return status;
}

int s3ttv_get_state(s3ttv_ctx *ctx, int which, float *dst) {
  if (!ctx) return S3TTV_EINVAL;
  if (!ctx->ready) return fail(ctx, S3TTV_ESTATE, "no problem set up");
  if (!dst) return fail(ctx, S3TTV_EINVAL, "dst is NULL");
  DeviceGuard g(ctx->device);
  int rc;
  switch (which) {
    case S3TTV_STATE_U: rc = store_cube(ctx, ctx->u, dst, nullptr); break;
    case S3TTV_STATE_S: rc = store_cube(ctx, ctx->s, dst, nullptr); break;
    case S3TTV_STATE_T: rc = store_cube(ctx, ctx->t[ctx->parity], dst, nullptr); break;
    case S3TTV_STATE_Y2: rc = store_cube(ctx, ctx->y2, dst, nullptr); break;
    case S3TTV_STATE_Y3: rc = store_cube(ctx, ctx->d, dst, &ctx->sc->c3); break;
    case S3TTV_STATE_Y: rc = store_Y(ctx, dst); break;
    default: return fail(ctx, S3TTV_EINVAL, "unknown state %d", which);
  }
  if (rc) return rc;
  CU(cudaStreamSynchronize(ctx->stream));
  return S3TTV_OK;
}

int s3ttv_set_state(s3ttv_ctx *ctx, int which, const float *src) {
  if (!ctx) return S3TTV_EINVAL;
  if (!ctx->ready) return fail(ctx, S3TTV_ESTATE, "no problem set up");
  if (!src) return fail(ctx, S3TTV_EINVAL, "src is NULL");
  DeviceGuard g(ctx->device);
  int rc;
  switch (which) {
    case S3TTV_STATE_U: rc = load_cube(ctx, src, ctx->u, 1.f); break;
    case S3TTV_STATE_S: rc = load_cube(ctx, src, ctx->s, 1.f); break;
    case S3TTV_STATE_T: rc = load_cube(ctx, src, ctx->t[ctx->parity], 1.f); break;
    case S3TTV_STATE_Y2: rc = load_cube(ctx, src, ctx->y2, 1.f); break;
    case S3TTV_STATE_Y3:
      rc = load_cube(ctx, src, ctx->d, 1.f);
      if (!rc) {
        set_c3_kernel<<<1, 1, 0, ctx->stream>>>(ctx->sc, 1.0);
        CU(cudaGetLastError());
      }
      break;
    case S3TTV_STATE_Y:
      ctx->warm_valid = false;
      rc = load_Y(ctx, src);
      if (!rc && (ctx->reg == S3TTV_REG_SSTV || is_hsstv(ctx))) {  // SSTV, HSSTV: Z = the second-order pair
        CU(cudaMemcpyAsync(ctx->Zv[ctx->parity], ctx->Y, sizeof(float) * ctx->dm.Np, cudaMemcpyDeviceToDevice,
                           ctx->stream));
        CU(cudaMemcpyAsync(ctx->Zh[ctx->parity], ctx->Y + ctx->dm.Np, sizeof(float) * ctx->dm.Np,
                           cudaMemcpyDeviceToDevice, ctx->stream));
      } else if (!rc) {
        CU(launch_Z_from_Y(ctx->Y, ctx->Zv[ctx->parity], ctx->Zh[ctx->parity], ctx->dm, ctx->k, ctx->stream,
                           is_ssst(ctx) ? ctx->Zs[ctx->parity] : nullptr));
      }
      break;
    default: return fail(ctx, S3TTV_EINVAL, "unknown state %d", which);
  }
  if (rc) return rc;
  CU(cudaStreamSynchronize(ctx->stream));
  return S3TTV_OK;
}

int s3ttv_solve(s3ttv_ctx *ctx, const float *v, int N1, int N2, int N3, float eps, float alpha, float beta,
                float mu_min, float mu_max, int k, int max_iter, float tol, float *u, float *s, float *t,
                s3ttv_info *info) {
  const double t0 = now_s();
  if (info) memset(info, 0, sizeof(*info));
  if (!ctx) return S3TTV_EINVAL;
  if (!u) return fail(ctx, S3TTV_EINVAL, "u is NULL");
  if (max_iter < 1) return fail(ctx, S3TTV_EINVAL, "max_iter = %d must be >= 1", max_iter);
  if (!(tol >= 0.f) || !std::isfinite(tol)) return fail(ctx, S3TTV_EINVAL, "tol must be finite and >= 0");
  NvtxRange nr(ctx->nvtx, "s3ttv_solve");
  int rc = s3ttv_setup(ctx, v, N1, N2, N3, eps, alpha, beta, mu_min, mu_max, k);
  if (rc) {
    if (info) info->status = rc;
    return rc;
  }
  s3ttv_info it;
  const int st = s3ttv_iterate(ctx, max_iter, tol, &it);
  if (st < 0) {
    if (info) {
      *info = it;
      info->status = st;
    }
    return st;
  }
  DeviceGuard g(ctx->device);
  if ((rc = store_cube(ctx, ctx->u, u, nullptr))) return rc;
  if (s && (rc = store_cube(ctx, ctx->s, s, nullptr))) return rc;
  if (t && (rc = store_cube(ctx, ctx->t[ctx->parity], t, nullptr))) return rc;
  CU(cudaStreamSynchronize(ctx->stream));
  if (info) {
    *info = it;
    info->status = st;
    info->seconds = now_s() - t0;
  }
  return st;
}

namespace {

// Fork from ctx->stream into every member stream and join back (events owned by
// the caller), so work enqueued on the members orders after, and before, the
// work on ctx->stream.
struct ForkJoin {
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  ~ForkJoin() {
    if (fork) cudaEventDestroy(fork);
    for (cudaEvent_t e : join)
      if (e) cudaEventDestroy(e);
  }
  cudaError_t create(size_t n) {
    cudaError_t e = cudaEventCreateWithFlags(&fork, cudaEventDisableTiming);
    join.assign(n, nullptr);
    for (size_t i = 0; i < n && e == cudaSuccess; ++i) e = cudaEventCreateWithFlags(&join[i], cudaEventDisableTiming);
    return e;
  }
};

// Enqueue `passes` passes of every member (member i starting at parity par[i])
// between a fork from and a join into ctx->stream.
int enqueue_batch(s3ttv_ctx *ctx, int n, const std::vector<BdShape> &bd, const std::vector<int> &grid_e,
                  const std::vector<int> &par, int passes, ForkJoin &fj) {
  CU(cudaEventRecord(fj.fork, ctx->stream));
  for (int i = 0; i < n; ++i) {
    s3ttv_ctx *m = ctx->members[i];
    CU(cudaStreamWaitEvent(m->stream, fj.fork, 0));
    for (int c = 0; c < passes; ++c) {
      const int rc = enqueue_pass(m, par[i] ^ (c & 1), grid_e[i], bd[i], nullptr);
      if (rc) return fail(ctx, rc, "problem %d: %s", i, m->err);
    }
    CU(cudaEventRecord(fj.join[i], m->stream));
    CU(cudaStreamWaitEvent(ctx->stream, fj.join[i], 0));
  }
  return S3TTV_OK;
}

}  // namespace

// The work lists of a batched solve's block duals: for each block side k in the
// batch, the problems with that k (their BlockDualArgs and running first-block
// offsets), for both parities of the Z buffers; one persistent launch per k.
struct BatchGroup {
  int k = 0, offset = 0, count = 0, grid = 0;  // items [offset, offset + count) of a parity's list
  long long total = 0;                         // blocks of the group's problems
};
struct BatchPlan {
  int n_items = 0;
  std::vector<BatchGroup> groups;
};

// Every member's block duals can join one work list: the streaming k <= 5 form
// of a regulariser with blocks (S3TTV or STV), all members at the same parity.
bool worklist_eligible(s3ttv_ctx *ctx, int n, const std::vector<BdShape> &bd, const std::vector<int> &par) {
  for (int i = 0; i < n; ++i) {
    const s3ttv_ctx *m = ctx->members[i];
    if (bd[i].large || bd[i].v.tc != 2 || par[i] != par[0]) return false;
    if (m->reg != S3TTV_REG_S3TTV && m->reg != S3TTV_REG_STV) return false;
  }
  return true;
}

int build_worklist(s3ttv_ctx *ctx, int n, const std::vector<BdShape> &bd, BatchPlan *plan) {
  std::vector<BatchDual> host;
  plan->groups.clear();
  for (int p = 0; p < 2; ++p) {
    for (int k = 1; k <= kMaxSmallK; ++k) {
      BatchGroup g;
      g.k = k;
      g.offset = (int)host.size() - p * plan->n_items;
      for (int i = 0; i < n; ++i) {
        s3ttv_ctx *m = ctx->members[i];
        if (m->k != k) continue;
        BatchDual it;
        it.a = make_bd_args(m, p, bd[i]);
        it.first = g.total;
        g.total += m->dm.P;
        host.push_back(it);
        ++g.count;
      }
      if (p == 0 && g.count) {
        int per_sm = 0;
        const cudaError_t e = block_dual_batch_prepare(k, &per_sm);
        if (e != cudaSuccess) return fail(ctx, S3TTV_ECUDA, "batched block dual, k = %d: %s", k, cudaGetErrorString(e));
        long long grid = (long long)ctx->num_sms * (per_sm > 0 ? per_sm : 1);
        const long long rounds = (g.total + block_dual_group() - 1) / block_dual_group();
        g.grid = (int)(grid < rounds ? grid : rounds);
        plan->groups.push_back(g);
      }
    }
    if (p == 0) plan->n_items = (int)host.size();
  }
  const size_t bytes = host.size() * sizeof(BatchDual);
  if (ctx->cap_items < bytes) {
    if (ctx->batch_items) {
      cudaFree(ctx->batch_items);
      ctx->bytes -= ctx->cap_items;
      ctx->batch_items = nullptr;
      ctx->cap_items = 0;
    }
    int rc = dmalloc(ctx, (void **)&ctx->batch_items, bytes);
    if (rc) return rc;
    ctx->cap_items = bytes;
  }
  CU(cudaMemcpyAsync(ctx->batch_items, host.data(), bytes, cudaMemcpyHostToDevice, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  return S3TTV_OK;
}

// Enqueue `passes` passes of every member: each pass's steps before the block
// duals on the members' own streams, then the block duals of all members in
// one work-list launch per block side on ctx->stream, then the steps after
// them on the members' streams again.
int enqueue_batch_worklist(s3ttv_ctx *ctx, int n, const std::vector<BdShape> &bd, const std::vector<int> &grid_e,
                           const std::vector<int> &par, int passes, ForkJoin &fj, const BatchPlan &plan) {
  for (int c = 0; c < passes; ++c) {
    for (int half = 1; half <= 2; ++half) {
      CU(cudaEventRecord(fj.fork, ctx->stream));
      for (int i = 0; i < n; ++i) {
        s3ttv_ctx *m = ctx->members[i];
        CU(cudaStreamWaitEvent(m->stream, fj.fork, 0));
        const int rc = enqueue_pass(m, par[i] ^ (c & 1), grid_e[i], bd[i], nullptr, half);
        if (rc) return fail(ctx, rc, "problem %d: %s", i, m->err);
        CU(cudaEventRecord(fj.join[i], m->stream));
        CU(cudaStreamWaitEvent(ctx->stream, fj.join[i], 0));
      }
      if (half == 1) {
        const int p = (par[0] ^ c) & 1;
        for (const BatchGroup &g : plan.groups) {
          CU(launch_block_dual_batch(g.k, ctx->batch_items + (size_t)p * plan.n_items + g.offset, g.count, g.total,
                                     g.grid, ctx->stream));
          ctx->launches += 1;
        }
      }
    }
  }
  return S3TTV_OK;
}

int s3ttv_solve_batched(s3ttv_ctx *ctx, int n, const s3ttv_problem *problems, int max_iter, float tol,
                        s3ttv_info *infos) {
  const double t0 = now_s();
  if (!ctx) return S3TTV_EINVAL;
  NvtxRange nr(ctx->nvtx, "s3ttv_solve_batched");
  if (n < 1) return fail(ctx, S3TTV_EINVAL, "n = %d must be >= 1", n);
  if (infos) memset(infos, 0, sizeof(*infos) * (size_t)n);
  if (!problems) return fail(ctx, S3TTV_EINVAL, "problems is NULL");
  if (max_iter < 1) return fail(ctx, S3TTV_EINVAL, "max_iter = %d must be >= 1", max_iter);
  if (!(tol >= 0.f) || !std::isfinite(tol)) return fail(ctx, S3TTV_EINVAL, "tol must be finite and >= 0");
  for (int i = 0; i < n; ++i)
    if (!problems[i].u) {
      if (infos) infos[i].status = S3TTV_EINVAL;
      return fail(ctx, S3TTV_EINVAL, "problem %d: u is NULL", i);
    }
  DeviceGuard g(ctx->device);
  while ((int)ctx->members.size() < n) {
    s3ttv_ctx *m = nullptr;
    const int rc = s3ttv_create(&m, ctx->device, nullptr);
    if (rc) return fail(ctx, rc, "creating the workspace of problem %zu failed", ctx->members.size());
    ctx->members.push_back(m);
  }
  std::vector<BdShape> bd(n);
  std::vector<int> grid_e(n), par(n, 0), iter0(n, 0);
  for (int i = 0; i < n; ++i) {
    s3ttv_ctx *m = ctx->members[i];
    m->step_policy = ctx->step_policy;
    m->jacobi_max_sweeps = ctx->jacobi_max_sweeps;
    m->jacobi_tol = ctx->jacobi_tol;
    m->jacobi_polish = ctx->jacobi_polish;
    m->first_order = ctx->first_order;
    m->tensor_cores = ctx->tensor_cores;
    m->warm_start = ctx->warm_start;
    m->layout = ctx->layout;
    m->open_s = ctx->open_s;
    m->reg = ctx->reg;
    m->hsstv_omega = ctx->hsstv_omega;
    m->fp64_fallback = ctx->fp64_fallback;
    m->profile = false;
    const s3ttv_problem &p = problems[i];
    int rc = s3ttv_setup(m, p.v, p.N1, p.N2, p.N3, p.eps, p.alpha, p.beta, p.mu_min, p.mu_max, p.k);
    if (!rc) rc = block_dual_shape(m, m->dm, m->k, &bd[i]);
    if (!rc) rc = ensure_rows(m, bd[i]);
    if (rc) {
      if (infos) infos[i].status = rc;
      return fail(ctx, rc, "problem %d: %s", i, m->err);
    }
    grid_e[i] = elementwise_grid(m, m->dm.Np);
    begin_iterate_kernel<<<1, 1, 0, m->stream>>>(m->sc, max_iter, tol);
    CU(cudaGetLastError());
    m->launches += 1;
    if (m->warm_start && m->W) {
      // every block starts cold on a NaN marker, so every recorded pass may
      // take the stored rows as they stand (warm from the second pass on)
      CU(cudaMemsetAsync(m->W, 0xff, sizeof(float) * (size_t)m->dm.P * m->w_stride, m->stream));
      m->warm_valid = true;
    }
  }
  BatchPlan plan;
  const bool worklist = ctx->batch_worklist && worklist_eligible(ctx, n, bd, par);
  if (worklist) {
    for (int i = 0; i < n; ++i) CU(cudaStreamSynchronize(ctx->members[i]->stream));
    const int rcw = build_worklist(ctx, n, bd, &plan);
    if (rcw) return rcw;
  }

  // one chunk of passes of every problem, recorded as a graph (an even number
  // of passes returns every problem to its starting parity)
  const int chunk = (ctx->check_every + 1) & ~1;
  ForkJoin fj;
  CU(fj.create(n));
  auto enqueue = [&](int passes) {
    return worklist ? enqueue_batch_worklist(ctx, n, bd, grid_e, par, passes, fj, plan)
                    : enqueue_batch(ctx, n, bd, grid_e, par, passes, fj);
  };
  cudaGraphExec_t exec = nullptr;
  std::vector<long long> launches0(n), per_pass(n, kLaunchesPerPass);
  // the legacy default streams cannot be captured: then every chunk is enqueued
  const bool capturable = ctx->stream != nullptr && ctx->stream != cudaStreamLegacy && ctx->stream != cudaStreamPerThread;
  if (max_iter >= chunk && capturable) {
    for (int i = 0; i < n; ++i) launches0[i] = ctx->members[i]->launches;
    CU(cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal));
    int rc = enqueue(chunk);
    cudaGraph_t graph = nullptr;
    const cudaError_t ec = cudaStreamEndCapture(ctx->stream, &graph);
    if (rc) {
      if (graph) cudaGraphDestroy(graph);
      cudaGetLastError();
      return rc;
    }
    CU(ec);
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    cudaGraphDestroy(graph);
    CU(ei);
    for (int i = 0; i < n; ++i) {  // recorded, not run
      per_pass[i] = (ctx->members[i]->launches - launches0[i]) / chunk;
      ctx->members[i]->launches = launches0[i];
    }
  }
  std::vector<Scalars> hs(n);
  std::vector<double> finish(n, -1.0);  // host time at which each problem was seen stopped
  int enq = 0, rc = S3TTV_OK;
  while (enq < max_iter) {
    const int step = max_iter - enq >= chunk ? chunk : max_iter - enq;
    if (step == chunk && exec) {
      const cudaError_t e = cudaGraphLaunch(exec, ctx->stream);
      if (e != cudaSuccess) {
        rc = fail(ctx, S3TTV_ECUDA, "cudaGraphLaunch: %s", cudaGetErrorString(e));
        break;
      }
      for (int i = 0; i < n; ++i) ctx->members[i]->launches += per_pass[i] * chunk;
    } else {
      if ((rc = enqueue(step))) break;
      for (int i = 0; i < n; ++i) par[i] ^= step & 1;
    }
    enq += step;
    for (int i = 0; i < n; ++i) {
      const cudaError_t e = cudaMemcpyAsync(&hs[i], ctx->members[i]->sc, sizeof(Scalars), cudaMemcpyDeviceToHost,
                                            ctx->stream);
      if (e != cudaSuccess) rc = fail(ctx, S3TTV_ECUDA, "reading problem %d's scalars: %s", i, cudaGetErrorString(e));
    }
    if (rc) break;
    const cudaError_t e = cudaStreamSynchronize(ctx->stream);
    if (e != cudaSuccess) {
      rc = fail(ctx, S3TTV_ECUDA, "batched passes: %s", cudaGetErrorString(e));
      break;
    }
    bool all_done = true;
    const double now = now_s() - t0;
    for (int i = 0; i < n; ++i) {
      all_done = all_done && hs[i].done;
      if (hs[i].done && finish[i] < 0.0) finish[i] = now;
    }
    if (all_done) break;
  }
  if (exec) cudaGraphExecDestroy(exec);
  if (rc) return rc;
  // results: each problem's outputs on its own stream, then one wait
  int result = S3TTV_OK;
  for (int i = 0; i < n; ++i) {
    s3ttv_ctx *m = ctx->members[i];
    const int done_iters = hs[i].iter - iter0[i];
    m->parity = done_iters & 1;
    int status;
    if (hs[i].status == -4) {
      status = S3TTV_ENUMERIC;
      fail(m, S3TTV_ENUMERIC, "NaN or Inf after %d passes", done_iters);
    } else {
      status = hs[i].status == 1 ? S3TTV_OK : S3TTV_MAXITER;
    }
    if (status >= 0) {
      const s3ttv_problem &p = problems[i];
      int r = store_cube(m, m->u, p.u, nullptr);
      if (!r && p.s) r = store_cube(m, m->s, p.s, nullptr);
      if (!r && p.t) r = store_cube(m, m->t[m->parity], p.t, nullptr);
      if (r) status = r;
    }
    if (infos) {
      infos[i].status = status;
      infos[i].iters = done_iters;
      infos[i].converged = hs[i].status == 1;
      infos[i].jacobi_nonconverged = (int)hs[i].jacobi_fail;
      infos[i].jacobi_fallbacks = (int)hs[i].fb_total;
      infos[i].rel_change = hs[i].rel;
      infos[i].jacobi_sweeps =
          done_iters > 0 ? (double)hs[i].jacobi_sweeps / ((double)done_iters * m->dm.P) : 0.0;
      infos[i].first_order = done_iters > 0 ? (double)hs[i].fo_blocks / ((double)done_iters * m->dm.P) : 0.0;
    }
    if (status < 0 && result >= 0) result = fail(ctx, status, "problem %d: %s", i, m->err);
    else if (status == S3TTV_MAXITER && result == S3TTV_OK) result = S3TTV_MAXITER;
  }
  for (int i = 0; i < n; ++i) {
    const cudaError_t e = cudaStreamSynchronize(ctx->members[i]->stream);
    if (e != cudaSuccess && result >= 0) result = fail(ctx, S3TTV_ECUDA, "problem %d: %s", i, cudaGetErrorString(e));
  }
  const double secs = now_s() - t0;
  if (infos)  // per problem: until its stop rule was seen (to a chunk of passes), else the whole call
    for (int i = 0; i < n; ++i) infos[i].seconds = finish[i] >= 0.0 ? finish[i] : secs;
  return result;
}

int s3ttv_l1_ball(s3ttv_ctx *ctx, const float *x, float *out, long long n, double radius, double *tau_out) {
  if (!ctx) return S3TTV_EINVAL;
  if (n < 0) return fail(ctx, S3TTV_EINVAL, "n < 0");
  if (!(radius >= 0) || !std::isfinite(radius)) return fail(ctx, S3TTV_EINVAL, "radius must be finite and >= 0");
  if (n > 0 && (!x || !out)) return fail(ctx, S3TTV_EINVAL, "x and out are required");
  if (n == 0) {
    if (tau_out) *tau_out = 0.0;
    return S3TTV_OK;
  }
  DeviceGuard g(ctx->device);
  int rc = ensure_common(ctx);
  if (rc) return rc;
  const bool xd = is_device_ptr(x), od = is_device_ptr(out);
  // stage: [host copy of x][output]
  const size_t need = (xd ? 0 : (size_t)n) + (od ? 0 : (size_t)n);
  if (need && (rc = ensure_stage(ctx, need))) return rc;
  const float *xin = x;
  float *xout = out;
  if (!xd) {
    CU(cudaMemcpyAsync(ctx->stage, x, sizeof(float) * n, cudaMemcpyHostToDevice, ctx->stream));
    xin = ctx->stage;
  }
  if (!od) xout = ctx->stage + (xd ? 0 : n);
  CU(launch_init_scalars(ctx->sc, radius, 0.0, ctx->stream));
  L1Args la;
  la.x[0] = xin;
  la.x[1] = xin;
  la.n = n;
  la.nprob = 1;
  la.sc = ctx->sc;
  la.hcnt = ctx->hcnt;
  la.hsum = ctx->hsum;
  const int grid = elementwise_grid(ctx, n);
  for (int level = 1; level <= 3; ++level) {
    CU(launch_l1_hist(la, level, grid, ctx->stream));
    CU(launch_l1_scan(la, level, ctx->stream));
  }
  CU(launch_soft_threshold(xin, xout, n, ctx->sc, 0, ctx->stream));
  if (!od) CU(cudaMemcpyAsync(out, xout, sizeof(float) * n, cudaMemcpyDeviceToHost, ctx->stream));
  Scalars hs;
  CU(cudaMemcpyAsync(&hs, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (tau_out) *tau_out = (double)hs.l1[0].tau;
  ctx->ready = false;  // the scalars of any set-up problem were overwritten
  return S3TTV_OK;
}

int s3ttv_block_dual(s3ttv_ctx *ctx, float *Y, const float *ubar, float *Zv, float *Zh, int N1, int N2, int N3,
                     int k, float gamma_Y, s3ttv_info *info) {
  if (info) memset(info, 0, sizeof(*info));
  if (!ctx) return S3TTV_EINVAL;
  NvtxRange nr(ctx->nvtx, "s3ttv_block_dual");
  if (!Y || !ubar || !Zv || !Zh) return fail(ctx, S3TTV_EINVAL, "Y, ubar, Zv and Zh are required");
  if (k < 1 || N1 < k || N2 < k || N3 < 1) return fail(ctx, S3TTV_EINVAL, "need N1, N2 >= k >= 1 and N3 >= 1");
  if (!(gamma_Y > 0.f) || !std::isfinite(gamma_Y)) return fail(ctx, S3TTV_EINVAL, "gamma_Y must be > 0");
  if (ctx->reg == S3TTV_REG_SSTV || is_hsstv(ctx))
    return fail(ctx, S3TTV_EUNSUPPORTED, "SSTV and HSSTV have no block duals");
  if (is_ssst(ctx)) return fail(ctx, S3TTV_EUNSUPPORTED, "SSST's block duals run inside the solver only");
  if (k > kMaxK) return fail(ctx, S3TTV_EUNSUPPORTED, "k = %d: this library supports k <= %d", k, kMaxK);
  DeviceGuard g(ctx->device);
  const Dims dm = make_dims(N1, N2, N3);
  int rc;
  BdShape bd;
  if ((rc = block_dual_shape(ctx, dm, k, &bd))) return rc;
  ctx->ready = false;
  if ((rc = ensure_problem_buffers(ctx, dm, k))) return rc;
  if ((rc = ensure_rows(ctx, bd))) return rc;
  ctx->dm = dm;
  ctx->k = k;
  if ((rc = load_Y(ctx, Y))) return rc;
  if ((rc = load_cube(ctx, ubar, ctx->ubar, 1.f))) return rc;
  CU(cudaMemsetAsync(ctx->Zv[0], 0, sizeof(float) * dm.Np, ctx->stream));
  CU(cudaMemsetAsync(ctx->Zh[0], 0, sizeof(float) * dm.Np, ctx->stream));
  CU(launch_init_scalars(ctx->sc, 0.0, 0.0, ctx->stream));
  CU(launch_xfield(ctx->ubar, ctx->Fv, ctx->Fh, dm, elementwise_grid(ctx, dm.Np), ctx->stream, ctx->open_s,
                   ctx->reg == S3TTV_REG_STV));
  BlockDualArgs ba;
  ba.Y = ctx->Y;
  ba.Fv = ctx->Fv;
  ba.Fh = ctx->Fh;
  ba.Zv = ctx->Zv[0];
  ba.Zh = ctx->Zh[0];
  ba.dm = dm;
  ba.gY = gamma_Y;
  ba.rs = bd.rs;
  ba.max_sweeps = ctx->jacobi_max_sweeps;
  ba.tol = ctx->jacobi_tol;
  ba.polish = jacobi_polish_for(ctx);
  ba.fo_tol = bd.large ? 0.f : ctx->first_order;
  ba.sc = ctx->sc;
  ba.W = nullptr;
  ba.w_stride = 0;
  ba.warm = 0;
  const bool fb = ctx->fp64_fallback && bd.fb_smem > 0;
  ba.fb_list = fb ? ctx->fb_list : nullptr;
  ba.fb_cap = fb ? ctx->fb_cap : 0;
  ba.rows = ctx->rows;
  ba.rows_cap = ctx->cap_rows / sizeof(float);
  if (bd.large) CU(launch_block_dual_large(ba, k, ctx->layout == S3TTV_LAYOUT_STACKED, bd.grid, bd.smem, ctx->stream));
  else CU(launch_block_dual(ba, bd.v, bd.grid, bd.smem, ctx->stream));
  if (fb)
    CU(launch_fallback(ba, k, ctx->layout == S3TTV_LAYOUT_STACKED, row_parts(ctx), ctx->num_sms, bd.fb_smem,
                       ctx->stream));
  if ((rc = store_Y(ctx, Y))) return rc;
  if ((rc = store_cube(ctx, ctx->Zv[0], Zv, nullptr))) return rc;
  if ((rc = store_cube(ctx, ctx->Zh[0], Zh, nullptr))) return rc;
  Scalars hs;
  CU(cudaMemcpyAsync(&hs, ctx->sc, sizeof(Scalars), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (info) {
    info->jacobi_nonconverged = (int)hs.jacobi_fail;
    info->jacobi_fallbacks = (int)hs.fb_total;
    info->jacobi_sweeps = (double)hs.jacobi_sweeps / (double)dm.P;
    info->first_order = (double)hs.fo_blocks / (double)dm.P;
  }
  return S3TTV_OK;
}

int s3ttv_tuned_form(const s3ttv_ctx *ctx, int *tensor_cores, int *ctas_per_sm) {
  if (!ctx || !tensor_cores || !ctas_per_sm) return S3TTV_EINVAL;
  *tensor_cores = ctx->tuned_tc;
  *ctas_per_sm = ctx->tuned_tc >= 0 ? ctx->tuned_minb : 0;
  return S3TTV_OK;
}

int s3ttv_objective(s3ttv_ctx *ctx, const float *u, int N1, int N2, int N3, int k, double *value) {
  if (!ctx) return S3TTV_EINVAL;
  if (!u || !value) return fail(ctx, S3TTV_EINVAL, "u and value are required");
  if (k < 1 || N1 < k || N2 < k || N3 < 1) return fail(ctx, S3TTV_EINVAL, "need N1, N2 >= k >= 1 and N3 >= 1");
  const int stacked = ctx->layout == S3TTV_LAYOUT_STACKED;
  if (k > (stacked || is_ssst(ctx) ? kMaxStackedK : kMaxK))
    return fail(ctx, S3TTV_EUNSUPPORTED, "k = %d: this library supports k <= %d", k,
                stacked || is_ssst(ctx) ? kMaxStackedK : kMaxK);
  if (is_ssst(ctx) && (stacked || ctx->open_s))
    return fail(ctx, S3TTV_EUNSUPPORTED, "SSST takes the paper layout and the periodic spectral boundary");
  DeviceGuard g(ctx->device);
  int rc;
  const long long N = (long long)N1 * N2 * N3;
  const float *du = u;
  if (!is_device_ptr(u)) {
    if ((rc = ensure_stage(ctx, (size_t)N))) return rc;
    CU(cudaMemcpyAsync(ctx->stage, u, sizeof(float) * N, cudaMemcpyHostToDevice, ctx->stream));
    du = ctx->stage;
  }
  if ((rc = ensure_macc(ctx, 2))) return rc;
  CU(cudaMemsetAsync(ctx->macc, 0, 2 * sizeof(double), ctx->stream));
  unsigned *nonconv = reinterpret_cast<unsigned *>(ctx->macc + 1);
  int dev_max = 0;
  CU(cudaDeviceGetAttribute(&dev_max, cudaDevAttrMaxSharedMemoryPerBlockOptin, ctx->device));
  if (objective_smem_bytes(k, stacked) + 2048 > (size_t)dev_max)
    return fail(ctx, S3TTV_EUNSUPPORTED, "k = %d needs %zu bytes of shared memory", k, objective_smem_bytes(k, stacked));
  if (ctx->reg == S3TTV_REG_SSTV)
    CU(launch_sstv_l1(du, N1, N2, N3, ctx->macc, ctx->num_sms * 8, ctx->stream));
  else if (is_hsstv(ctx))
    CU(launch_hsstv_norm(du, N1, N2, N3, ctx->hsstv_omega, ctx->reg == S3TTV_REG_HSSTV2, ctx->macc, ctx->num_sms * 8,
                         ctx->stream));
  else
    CU(launch_objective(du, N1, N2, N3, k, stacked, ctx->open_s, ctx->reg == S3TTV_REG_STV || is_ssst(ctx),
                        ctx->macc, nonconv, ctx->num_sms * 4, ctx->stream, row_parts(ctx)));
  double h[2] = {0.0, 0.0};
  CU(cudaMemcpyAsync(h, ctx->macc, 2 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  unsigned nc;
  memcpy(&nc, &h[1], sizeof(nc));
  if (nc) return fail(ctx, S3TTV_ENUMERIC, "%u blocks did not converge in the FP64 Jacobi", nc);
  if (!std::isfinite(h[0])) return fail(ctx, S3TTV_ENUMERIC, "u is not finite");
  *value = h[0];
  return S3TTV_OK;
}

int s3ttv_quality(s3ttv_ctx *ctx, const float *u, const float *ref, int N1, int N2, int N3, int trim,
                  double *mpsnr, double *mssim, double *sam_mean, float *sam_map) {
  if (!ctx) return S3TTV_EINVAL;
  if (!u || !ref) return fail(ctx, S3TTV_EINVAL, "u and ref are required");
  if (N1 < 1 || N2 < 1 || N3 < 1 || trim < 0) return fail(ctx, S3TTV_EINVAL, "need N1, N2, N3 >= 1 and trim >= 0");
  const int r = kSsimTaps / 2;
  if (mssim && (N1 <= 2 * r || N2 <= 2 * r))
    return fail(ctx, S3TTV_EINVAL, "MSSIM needs N1, N2 >= %d (one whole %dx%d window)", 2 * r + 1, 2 * r + 1,
                2 * r + 1);
  DeviceGuard g(ctx->device);
  int rc;
  if ((rc = ensure_common(ctx))) return rc;
  const long long P = (long long)N1 * N2, N = P * N3;
  const int b0 = N3 > 2 * trim ? trim : 0, nb = N3 > 2 * trim ? N3 - 2 * trim : N3;
  const bool ud = is_device_ptr(u), rd = is_device_ptr(ref), md = !sam_map || is_device_ptr(sam_map);
  if (!ud || !rd || !md) {
    if ((rc = ensure_stage(ctx, (size_t)(2 * N + P)))) return rc;
  }
  const float *du = u, *dr = ref;
  if (!ud) {
    CU(cudaMemcpyAsync(ctx->stage, u, sizeof(float) * N, cudaMemcpyHostToDevice, ctx->stream));
    du = ctx->stage;
  }
  if (!rd) {
    CU(cudaMemcpyAsync(ctx->stage + N, ref, sizeof(float) * N, cudaMemcpyHostToDevice, ctx->stream));
    dr = ctx->stage + N;
  }
  float *dmap = sam_map ? (md ? sam_map : ctx->stage + 2 * N) : nullptr;
  if ((rc = ensure_macc(ctx, (size_t)2 * N3 + 1))) return rc;
  CU(cudaMemsetAsync(ctx->macc, 0, sizeof(double) * (2 * N3 + 1), ctx->stream));
  const int grid = ctx->num_sms * 8;
  if (mpsnr) CU(launch_band_sqerr(du, dr, P, N3, ctx->macc, grid, ctx->stream));
  if (mssim) CU(launch_ssim(du, dr, N1, N2, N3, b0, nb, ctx->macc + N3, grid, ctx->stream));
  if (sam_mean || sam_map) CU(launch_sam(du, dr, P, N3, dmap, ctx->macc + 2 * N3, grid, ctx->stream));
  if (sam_map && !md)
    CU(cudaMemcpyAsync(sam_map, dmap, sizeof(float) * P, cudaMemcpyDeviceToHost, ctx->stream));
  std::vector<double> h((size_t)2 * N3 + 1);
  CU(cudaMemcpyAsync(h.data(), ctx->macc, sizeof(double) * h.size(), cudaMemcpyDeviceToHost, ctx->stream));
  CU(cudaStreamSynchronize(ctx->stream));
  if (mpsnr) {
    double s = 0.0;
    for (int b = b0; b < b0 + nb; ++b) s += h[b] > 0.0 ? 10.0 * log10((double)P / h[b]) : INFINITY;
    *mpsnr = s / nb;
  }
  if (mssim) {
    const double npix = (double)(N1 - 2 * r) * (N2 - 2 * r);
    double s = 0.0;
    for (int b = 0; b < nb; ++b) s += h[N3 + b] / npix;
    *mssim = s / nb;
  }
  if (sam_mean) *sam_mean = h[2 * N3] / (double)P;
  return S3TTV_OK;
}

}  // extern "C"
