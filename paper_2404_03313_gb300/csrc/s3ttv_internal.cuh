// Internal declarations shared by the CUDA translation units of libs3ttv.
//
// Internal layout.  Every cube lives as [N1][N2][N3p] with N3p = N3 rounded up to
// a multiple of 4, so each pixel's spectrum starts on a 16-byte boundary and the
// kernels can move float4s; the padding bands are kept at exactly zero.  The
// block dual Y lives as [L][k*k][2][N3p]: per block row, the N3p vertical
// differences (eq. SSST columns 2b) followed by the N3p horizontal ones (columns
// 2b+1).  A column permutation of a block does not change its singular values,
// so this is the same prox.  The fidelity dual is stored as y3 = c3 * d with a
// device scalar c3 and a cube d (see dual_kernel).
#pragma once
#include <cuda_runtime.h>
#include <type_traits>
#include <stdint.h>

namespace s3ttv {

constexpr int kHistBins = 2048;  // bins of the widest radix level
constexpr unsigned kFull = 0xffffffffu;

struct Dims {
  int N1, N2, N3, N3p;
  long long P;   // pixels N1*N2 (= number of blocks L)
  long long Np;  // P * N3p, elements of an internal cube
};

// One l1-ball projection being solved by radix selection over the bits of |z|.
struct L1State {
  double radius;
  double S_above;               // sum of |z| over bins above the current prefix
  unsigned long long C_above;   // count of those
  unsigned prefix;              // bits of |z| fixed so far
  int mode;                     // 0 searching, 1 inside the ball (tau 0), 2 radius 0, 3 found
  float tau;                    // soft threshold once mode != 0 (rounded)
  float tau_lo;                 // tau - (double)tau, so tau + tau_lo carries ~48 bits
};

// Device-resident scalars of one solve.
struct Scalars {
  L1State l1[2];       // [0] sparse noise s, [1] stripe noise t
  double c3;           // y3 = c3 * d
  double rel;          // relative change of the last pass
  int iter;            // passes completed since setup
  int iter_limit;      // stop when iter reaches this
  int done;            // set once the stop rule or the cap fired
  int status;          // 0 running, 1 converged, 2 cap, -4 numeric
  unsigned jacobi_fail;  // blocks left with an unconverged eigen-solve
  float tol;
  unsigned long long jacobi_sweeps;  // sweeps summed over blocks (statistics)
  unsigned fb_count;  // blocks queued for the FP64 re-solve in this pass (reset by the primal step)
  unsigned fb_total;  // blocks re-solved in FP64 since the last s3ttv_iterate began
  unsigned long long fo_blocks;  // blocks whose clip came from the first-order update (statistics)
};

// Radix levels over the 31 magnitude bits of a float.
__host__ __device__ inline int l1_level_bits(int level) { return level == 3 ? 9 : 11; }
__host__ __device__ inline int l1_level_shift(int level) { return level == 1 ? 20 : (level == 2 ? 9 : 0); }

// Soft threshold sign(z) max(|z| - tau, 0); tau = +inf gives 0.  The threshold
// comes as a float pair tau + tau_lo: when |z| and tau are within a factor of two
// |z| - tau is exact in FP32, so the one rounding left is that of subtracting
// tau_lo, and the result keeps full relative precision even when |z| - tau is
// many orders of magnitude below |z|.
__device__ __forceinline__ float soft_threshold(float z, float tau, float tau_lo) {
  const float m = (fabsf(z) - tau) - tau_lo;
  return m > 0.f ? copysignf(m, z) : 0.f;
}

// ---- launch wrappers (each returns the launch error) ----
struct PrimalArgs {
  const float *Zv, *Zh;   // sum_l P_l^T Y_l of the current Y
  float *Znv, *Znh;       // next accumulation target, zeroed here
  float *u, *ubar;        // u is updated in place, ubar = 2u+ - u
  const float *s, *t, *y2, *d;
  float *zs, *zt;         // pre-projection arguments of steps 3 and 4
  Dims dm;
  float gu, gs, gt, lo, hi;
  Scalars *sc;
  double *part;           // [2][grid]: sum (u+ - u)^2, sum u^2
  unsigned *hcnt;         // [2][kHistBins]
  double *hsum;           // [2][kHistBins]
  int no_ds;              // 1: the dual term is D^T Z (STV's first-order tensors), no D_s^T
  const float *Z1v = nullptr, *Z1h = nullptr;  // HSSTV: first-order dual pair, adds w1 D^T Z1
  float w1 = 0.f;
  const float *Zs = nullptr;  // SSST: the spectral part, adds D_s^T Zs
  float *Zns = nullptr;       // its next accumulation target, zeroed here
};
cudaError_t launch_primal(const PrimalArgs &a, int grid, cudaStream_t st);

struct DualArgs {
  const float *zs, *zt, *s_old, *t_old, *ubar, *v;
  float *s_new, *t_new, *y2, *d;
  Dims dm;
  float g2, g3;
  Scalars *sc;
  double *part;           // [grid]: sum d^2
};
cudaError_t launch_dual(const DualArgs &a, int grid, cudaStream_t st);

struct FinalizeArgs {
  Scalars *sc;
  const double *part_primal;  // [2][grid_p]
  int grid_p;
  const double *part_dual;    // [grid_d]
  int grid_d;
  double eps;
  double g3;
};
cudaError_t launch_finalize(const FinalizeArgs &a, cudaStream_t st);

// l1-ball radix selection: histogram pass over up to two vectors and the scan
// that narrows the threshold one level.
struct L1Args {
  const float *x[2];
  long long n;            // elements of each vector (both the same length)
  int nprob;              // 1 or 2
  Scalars *sc;
  unsigned *hcnt;         // [2][kHistBins]
  double *hsum;           // [2][kHistBins]
};
cudaError_t launch_l1_hist(const L1Args &a, int level, int grid, cudaStream_t st);
cudaError_t launch_l1_scan(const L1Args &a, int level, cudaStream_t st);
cudaError_t launch_soft_threshold(const float *x, float *out, long long n, const Scalars *sc,
                                  int prob, cudaStream_t st);

// Block dual (Alg. 1 steps 8-11) for all blocks.
struct BlockDualArgs {
  float *Y;               // [L][k*k][2][N3p], in place
  const float *Fv, *Fh;   // D_v D_s ubar and D_h D_s ubar (internal cubes)
  float *Zv, *Zh;         // accumulated with +=
  Dims dm;
  float gY;
  int rs;                 // shared-memory row stride (floats) of the block copies
  int max_sweeps;
  float tol;              // a sweep with a pair less orthogonal than this is followed by another
  float polish;           // (<= tol) pairs less orthogonal than this are rotated
  float fo_tol;           // bound on the remainder of the first-order clip (0: path off; k <= 5 kernel)
  Scalars *sc;            // done flag and the non-convergence counter
  float *W;               // per-block warm-start rows [L][w_stride] (may be null)
  long long w_stride;     // floats per block in W (>= NPOS * k*k)
  int warm;               // 1: start from the rows stored in W
  const float *Fs = nullptr;  // SSST's third part D_s ubar (per-CTA kernel, three parts)
  float *Zs = nullptr;        // and its accumulation
  // FP64 re-solve queue (fallback.cu): a block whose FP32 eigen-solve reaches
  // the sweep cap is listed here (up to fb_cap), left as Y' and not added to Z;
  // null: no queue, such blocks are applied as they stand
  int *fb_list = nullptr;
  int fb_cap = 0;
  // blocks above kMaxSmemRows rows: the per-CTA global rows of the two n x n
  // matrices (block_dual_large_rows_floats() floats per CTA of the grid);
  // rows_cap floats in all (the launcher refuses a grid they do not cover)
  float *rows = nullptr;
  size_t rows_cap = 0;
};
// floats per block of the warm-start rows
long long block_dual_w_stride(int k);
// FP64 re-solve of the queued blocks (fallback.cu); n = rows of a block matrix
size_t fallback_smem_bytes(int n);
cudaError_t fallback_prepare(size_t smem_bytes);
cudaError_t launch_fallback(const BlockDualArgs &a, int k, int stacked, int parts, int grid, size_t smem,
                            cudaStream_t st);
// Kernel variant: block side k (1..5), minb = 5 or 4 (CTAs per SM its register
// budget is sized for), tc = 1 for the Gram and the apply on tensor cores (three
// TF32 products per FP32 product), 0 for FP32 CUDA cores.
struct BdVariant {
  int k = 0;
  int minb = 4;
  int tc = 0;
};
// Row strides (floats) of the shared block copies for N3p bands.
int block_dual_row_stride(int N3p);
size_t block_dual_smem_bytes(const BdVariant &v, int N3p);
int block_dual_threads();
// blocks one CTA of the block-dual kernel takes at a time
int block_dual_group();
// All return cudaErrorInvalidValue for an unsupported variant.
cudaError_t launch_block_dual(const BlockDualArgs &a, const BdVariant &v, int grid, size_t smem, cudaStream_t st);
// The batched solve's block duals (streaming form, k <= 5): one persistent
// launch per block side k over a work list of the blocks of every problem with
// that k.
struct BatchDual {
  BlockDualArgs a;   // the problem's arguments (its own Y, F, Z, W, sizes, scalars)
  long long first;   // its first entry in the work list (a running sum of N1 * N2)
};
cudaError_t block_dual_batch_prepare(int k, int *ctas_per_sm);
cudaError_t launch_block_dual_batch(int k, const BatchDual *items, int n, long long total, int grid, cudaStream_t st);
bool block_dual_has(const BdVariant &v);  // this variant is compiled into the library
// Larger blocks, k = kMinLargeK..kMaxLargeK (block_dual_large.cu): one CTA of
// block_dual_large_threads() threads per block at a time, FP32 CUDA cores.
// The same kernel also runs the stacked layout (2 k^2 rows of N3 bands, rows 2r
// and 2r + 1 the vertical and horizontal differences of window pixel r) for
// k = 1..kMaxStackedK; the block memory [L][k^2][2][N3p] is the same.  Blocks
// of more than kMaxSmemRows rows (k = 13..16) keep their two n x n matrices in a
// global scratch of block_dual_large_rows_floats() floats per CTA (L2-resident).
constexpr int kMinLargeK = 6, kMaxLargeK = 16, kMaxStackedK = 8, kMaxSmemRows = 144;
constexpr int kMaxSmallK = kMinLargeK - 1;  // the k <= 5 kernels (block_dual.cu)
// parts = 3: SSST's rows [D_v u, D_h u, D_s u] (paper layout, k <= kMaxStackedK)
size_t block_dual_large_smem_bytes(int k, bool stacked, int parts = 2);
long long block_dual_large_w_stride(int k, bool stacked);
long long block_dual_large_w_stride(int k);  // paper layout
int block_dual_large_threads(int k, bool stacked, int parts = 2);
size_t block_dual_large_rows_floats(int k, bool stacked, int parts = 2);
cudaError_t block_dual_large_prepare(int k, bool stacked, size_t smem_bytes, int parts = 2);
cudaError_t block_dual_large_occupancy(int k, bool stacked, size_t smem_bytes, int *ctas_per_sm, int parts = 2);
cudaError_t launch_block_dual_large(const BlockDualArgs &a, int k, bool stacked, int grid, size_t smem,
                                    cudaStream_t st, int parts = 2);
cudaError_t block_dual_prepare(const BdVariant &v, size_t smem_bytes);
cudaError_t block_dual_occupancy(const BdVariant &v, size_t smem_bytes, int *ctas_per_sm);

// Layout conversion and small helpers.
cudaError_t launch_pad_cube(const float *src, float *dst, Dims dm, float scale, cudaStream_t st);
cudaError_t launch_unpad_cube(const float *src, float *dst, Dims dm, const double *scale_dev, cudaStream_t st);
cudaError_t launch_Y_to_internal(const float *ext, float *in, Dims dm, int k, cudaStream_t st, int stacked,
                                 int parts = 2);
cudaError_t launch_Y_to_external(const float *in, float *ext, Dims dm, int k, cudaStream_t st, int stacked,
                                 int parts = 2);
// Fv = D_v D_s ubar, Fh = D_h D_s ubar (Sec. II-A differences, periodic)
// open_s: the spectral difference stops at the last band (F's last band is 0)
// first_order: F = (D_v u, D_h u) (STV) instead of the second-order differences;
// with Fs as well, SSST's first-order parts (D_v u, D_h u, D_s u)
cudaError_t launch_xfield(const float *ubar, float *Fv, float *Fh, Dims dm, int grid, cudaStream_t st,
                         int open_s, int first_order, float *Fs = nullptr);
// SSTV's dual step: Y = clip(Y + gamma_Y D D_s ubar, -1, 1) on the cube pair
// (Yv, Yh), and Z = Y
cudaError_t launch_sstv_dual(const float *ubar, float *Yv, float *Yh, float *Zv, float *Zh, Dims dm, float gY,
                             int grid, cudaStream_t st);
// HSSTV's dual step on four cubes Y (second-order pair then omega-weighted
// first-order pair): l1 (l12 = 0) or per-voxel l1,2 (l12 = 1) conjugate prox
cudaError_t launch_hsstv_dual(const float *ubar, float *Y, float *Zv, float *Zh, Dims dm, float gY, float omega,
                              int l12, int grid, cudaStream_t st);
cudaError_t launch_Z_from_Y(const float *Y, float *Zv, float *Zh, Dims dm, int k, cudaStream_t st,
                            float *Zs = nullptr);
cudaError_t launch_init_scalars(Scalars *sc, double alpha, double beta, cudaStream_t st);

// evaluation (metrics.cu); plain [N1][N2][N3] cubes, FP64 sums
constexpr int kSsimTaps = 11;
cudaError_t launch_band_sqerr(const float *u, const float *ref, long long P, int N3, double *out, int grid,
                              cudaStream_t st);
cudaError_t launch_sam(const float *u, const float *ref, long long P, int N3, float *map, double *sum, int grid,
                       cudaStream_t st);
cudaError_t launch_ssim(const float *u, const float *ref, int N1, int N2, int N3, int b0, int nb, double *out,
                        int grid, cudaStream_t st);
size_t objective_smem_bytes(int k, int stacked);  // rows: k^2 or 2k^2
cudaError_t launch_objective(const float *u, int N1, int N2, int N3, int k, int stacked, int open_s,
                             int first_order, double *out, unsigned *nonconv, int grid, cudaStream_t st,
                             int parts = 2);
cudaError_t launch_sstv_l1(const float *u, int N1, int N2, int N3, double *out, int grid, cudaStream_t st);
cudaError_t launch_hsstv_norm(const float *u, int N1, int N2, int N3, double omega, int l12, double *out, int grid,
                              cudaStream_t st);


// ---------------------------------------------------------------------------
// FP32 products on the TF32 tensor cores (mma.sync m16n8k8), shared by both
// block-dual kernels.
// x ~ hi + lo with hi = x truncated to TF32 (low 13 mantissa bits cleared,
// |x - hi| < 2^-10 |x|) and lo = x - hi (exact in FP32) truncated to TF32 as
// well: |x - hi - lo| < 2^-20 |x|.  The TF32 tensor-core operands ignore the
// low 13 bits of their 32-bit registers (checked on GB300: every product of
// raw and of masked operands agreed bit for bit), so both parts go in
// unmasked: two instructions, the same products.
__device__ __forceinline__ void split_tf32(float x, unsigned &hi, unsigned &lo) {
  hi = __float_as_uint(x);
  lo = __float_as_uint(x - __uint_as_float(hi & 0xffffe000u));
}
// d += A B for one 16 x 8 x 8 tile, TF32 operands, FP32 accumulation (warp-wide).
__device__ __forceinline__ void mma_tf32(float (&d)[4], unsigned a0, unsigned a1, unsigned a2, unsigned a3,
                                         unsigned b0, unsigned b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k8.row.col.f32.tf32.tf32.f32 {%0, %1, %2, %3}, {%4, %5, %6, %7}, {%8, %9}, "
      "{%0, %1, %2, %3};\n"
      : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
      : "r"(a0), "r"(a1), "r"(a2), "r"(a3), "r"(b0), "r"(b1));
}
// d += A B with both operands split hi + lo: lo*hi + hi*lo + hi*hi (the lo*lo
// term, below 2^-20 of the product, is dropped), so the tile product keeps
// FP32-level accuracy (a few 2^-20 relative).  Product p of the three (0: lo*hi,
// 1: hi*lo, 2: hi*hi), in that order on every accumulator.  The call sites run
// p as their outermost loop over independent tiles, so consecutive products on
// one accumulator are several instructions apart instead of waiting out each
// other's latency (the same sums in the same order).
template <int p>
__device__ __forceinline__ void mma_3xtf32_part(float (&d)[4], const unsigned (&ah)[4], const unsigned (&al)[4],
                                                unsigned bh0, unsigned bh1, unsigned bl0, unsigned bl1) {
  if constexpr (p == 0) mma_tf32(d, al[0], al[1], al[2], al[3], bh0, bh1);
  else if constexpr (p == 1) mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bl0, bl1);
  else mma_tf32(d, ah[0], ah[1], ah[2], ah[3], bh0, bh1);
}
// F(integral_constant<int, p>) for p = 0, 1, 2
template <class F>
__device__ __forceinline__ void three_parts(const F &f) {
  f(std::integral_constant<int, 0>());
  f(std::integral_constant<int, 1>());
  f(std::integral_constant<int, 2>());
}

}  // namespace s3ttv
