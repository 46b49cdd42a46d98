// Learned warm start: a 3-D convolutional U-Net that maps the noisy cube v to an
// estimate of Alg. 1's primal variables (u, s, t), used to initialise the solver.
// The paper has no network (Alg. 1 starts from u = v, s = t = 0); the solver
// still decides the result, the network only moves its starting point.
//
// Network (3 levels, 32 / 64 / 128 channels; every conv is 3 x 3 x 3 with zero
// padding, bias and ReLU; pooling is the mean of 2 x 2 x 2 cells; upsampling is
// nearest):
//   e1a = conv(v)          e1b = conv(e1a)                      [full size, 32]
//   e2a = conv(pool(e1b))  e2b = conv(e2a)                      [half, 64]
//   ba  = conv(pool(e2b))  bb  = conv(ba)                       [quarter, 128]
//   d2a = conv(cat[up(bb), e2b])  d2b = conv(d2a)               [half, 64]
//   d1a = conv(cat[up(d2b), e1b]) d1b = conv(d1a)               [full size, 32]
//   h = Wh d1b + bh (1 x 1 x 1 to 3 channels); (u, s, t) = (v + h0, h1, h2).
// Training minimises the mean squared error against solver outputs with Adam.
//
// Precision: weights are used as BF16 (rounded from FP32 master copies held for
// Adam), activations and activation gradients are stored as BF16, every product
// accumulates in FP32, weight gradients accumulate in FP32, the loss in FP64.
//
// Layout: activations are channels-last, [B][D][H][W][C] (C fastest), so one
// voxel's channels are contiguous and a 32-channel slice is one 64-byte row.  A
// cube [N1][N2][N3] is the volume D = N1, H = N2, W = N3.
//
// Kernels.  The convolutions are implicit GEMMs on the tensor cores
// (mma.sync m16n8k16, BF16 in, FP32 accumulate), fed by cp.async gathers:
//  * conv_fwd_kernel: Y[p, o] = sum_{tap, c} X[p + delta_tap, c] Wt[o, tap, c]:
//    M = voxels (128 per CTA), N = output channels (32 or 64 per CTA), K = 27
//    taps x input channels in 32-channel steps; an input may be the channel
//    concatenation of a same-size tensor and a half-size one read through
//    nearest upsampling.  Epilogue: bias, ReLU, a ReLU mask (for backward).
//    The input gradient of a conv is the same kernel with the output gradient
//    as input and the weights transposed and mirrored, Wb[c, 26 - tap, o].
//  * conv_wgrad_kernel: dW[o, tap, c] = sum_p G[p, o] X[p + delta_tap, c]:
//    M = output channels, N = 32 input channels of one tap, K = voxels of one
//    chunk; fragments come from the voxel-major tiles through ldmatrix.trans;
//    partial sums are added into FP32 dW with atomics.
//  * the first layer (one input channel) and the head run on CUDA cores; the
//    first layer's weight gradient goes through an im2col of its 27 taps and
//    the tensor-core weight-gradient kernel.
#include <cuda_bf16.h>
#include <cuda_runtime.h>
#include <math.h>
#include <stdarg.h>
#include <stdint.h>
#include <stdio.h>
#include <string.h>

#include <new>

#include "s3ttv.h"

namespace {

typedef __nv_bfloat16 bf16;

constexpr int kLayers = 10;
constexpr int kCin[kLayers] = {1, 32, 32, 64, 64, 128, 192, 64, 96, 32};
constexpr int kCout[kLayers] = {32, 32, 64, 64, 128, 128, 64, 64, 32, 32};
constexpr int kHeadIn = 32, kHeadOut = 3;
constexpr long long kMaxVoxels = 1LL << 26;

struct Vol {
  int B, D, H, W;
};
__host__ __device__ inline int nvox(const Vol &g) { return g.B * g.D * g.H * g.W; }

struct LayerTable {
  long long woff[kLayers], boff[kLayers];
  int cin[kLayers], cout[kLayers];
  long long hw_off, hb_off, total;
};

LayerTable make_table() {
  LayerTable t;
  long long off = 0;
  for (int l = 0; l < kLayers; ++l) {
    t.cin[l] = kCin[l];
    t.cout[l] = kCout[l];
    t.woff[l] = off;
    off += 27LL * kCin[l] * kCout[l];
    t.boff[l] = off;
    off += kCout[l];
  }
  t.hw_off = off;
  off += kHeadIn * kHeadOut;
  t.hb_off = off;
  off += kHeadOut;
  t.total = off;
  return t;
}

// ---------------------------------------------------------------- PTX helpers
__device__ __forceinline__ void cp_async16(void *smem, const void *gmem, int src_bytes) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(smem);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16, %2;\n" ::"r"(s), "l"(gmem), "r"(src_bytes));
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
__device__ __forceinline__ void cp_async_wait1() { asm volatile("cp.async.wait_group 1;\n" ::); }

__device__ __forceinline__ void ldsm_x4(uint32_t r[4], const void *p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}
__device__ __forceinline__ void ldsm_x4_t(uint32_t r[4], const void *p) {
  const unsigned s = (unsigned)__cvta_generic_to_shared(p);
  asm volatile("ldmatrix.sync.aligned.m8n8.x4.trans.shared.b16 {%0,%1,%2,%3}, [%4];\n"
               : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3])
               : "r"(s));
}
// D = A B + D for a 16 x 16 (row) by 16 x 8 (col) BF16 tile, FP32 accumulate.
__device__ __forceinline__ void mma_bf16(float c[4], const uint32_t a[4], uint32_t b0, uint32_t b1) {
  asm volatile(
      "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 {%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, "
      "{%0,%1,%2,%3};\n"
      : "+f"(c[0]), "+f"(c[1]), "+f"(c[2]), "+f"(c[3])
      : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

__device__ __forceinline__ void decode(int p, const Vol &g, int &b, int &z, int &y, int &x) {
  x = p % g.W;
  int t = p / g.W;
  y = t % g.H;
  t /= g.H;
  z = t % g.D;
  b = t / g.D;
}

// 8 BF16 values <-> 8 floats through one 16-byte access
__device__ __forceinline__ void load8(const bf16 *p, float f[8]) {
  const uint4 u = *reinterpret_cast<const uint4 *>(p);
  const __nv_bfloat162 *h = reinterpret_cast<const __nv_bfloat162 *>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    const float2 t = __bfloat1622float2(h[i]);
    f[2 * i] = t.x;
    f[2 * i + 1] = t.y;
  }
}
__device__ __forceinline__ void store8(bf16 *p, const float f[8]) {
  uint4 u;
  __nv_bfloat162 *h = reinterpret_cast<__nv_bfloat162 *>(&u);
#pragma unroll
  for (int i = 0; i < 4; ++i) h[i] = __floats2bfloat162_rn(f[2 * i], f[2 * i + 1]);
  *reinterpret_cast<uint4 *>(p) = u;
}

// ---------------------------------------------------------------- conv forward
constexpr int kBK = 32;     // input channels per K step
constexpr int kAS = 40;     // shared row stride in bf16 (80 B: ldmatrix rows hit distinct banks)
constexpr int kStages = 3;  // cp.async pipeline depth

struct ConvArgs {
  const bf16 *x0;
  const bf16 *x1;
  const bf16 *w;       // [cout][27][c1 + c0]
  const float *bias;   // [cout] or null
  const bf16 *mask;    // [V][cout] or null: output zeroed where mask <= 0
  bf16 *y;             // [V][cout]
  int c0, c1, cout, relu;
  Vol g;
};

template <int BM, int BN>
constexpr int conv_smem_bytes() {
  return kStages * (BM + BN) * kAS * (int)sizeof(bf16);
}

// CTA tile BM voxels x BN output channels; (BM / 32) x (BN / 32) warps, each
// owning a 32 x 32 tile (2 m16 x 4 n8 fragments).  The K loop runs tap by tap
// and, within a tap, over 32-channel slices of the input; the voxel rows a
// thread gathers get their neighbour pointers once per tap.
template <int BM, int BN>
__global__ void __launch_bounds__((BM / 32) * (BN / 32) * 32) conv_fwd_kernel(ConvArgs a) {
  constexpr int WN = BN / 32;
  constexpr int NTH = (BM / 32) * WN * 32;
  constexpr int RPT = BM * 4 / NTH;  // 16-byte A pieces a thread copies per stage
  constexpr int AE = BM * kAS, BE = BN * kAS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16 *As = reinterpret_cast<bf16 *>(smem_raw);
  bf16 *Bs = As + kStages * AE;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp / WN, wn = warp % WN;
  const int V = nvox(a.g);
  const int m0 = blockIdx.x * BM, n0 = blockIdx.y * BN;
  const int cin = a.c0 + a.c1, nch = cin / kBK, ksteps = 27 * nch;
  const int q = tid & 3;
  // per gathered row: its voxel index, its index in the half-size grid, and a
  // mask of the volume faces it touches (bit 0/1: z = 0 / D-1, 2/3: y, 4/5: x,
  // 6: past the last voxel) plus its coordinate parities (bits 8-10: z, y, x)
  int vi[RPT], li[RPT], rm[RPT];
  const int D2 = a.g.D >> 1, H2 = a.g.H >> 1, W2 = a.g.W >> 1;
#pragma unroll
  for (int i = 0; i < RPT; ++i) {
    const int p = m0 + (tid >> 2) + i * (NTH / 4);
    int b, z, y, x;
    decode(p < V ? p : 0, a.g, b, z, y, x);
    vi[i] = p;
    li[i] = ((b * D2 + (z >> 1)) * H2 + (y >> 1)) * W2 + (x >> 1);
    rm[i] = (z == 0) | (z == a.g.D - 1) << 1 | (y == 0) << 2 | (y == a.g.H - 1) << 3 | (x == 0) << 4 |
            (x == a.g.W - 1) << 5 | (p >= V) << 6 | (z & 1) << 8 | (y & 1) << 9 | (x & 1) << 10;
  }
  // loader state: the tap and slice of the next stage to load; per tap the
  // faces it may not cross and the neighbour offset in the full-size grid
  int ltap = -1, lch = nch, forbid = 0, off0 = 0, dz = 0, dy = 0, dx = 0;
  auto load = [&](int buf) {
    if (lch == nch) {
      lch = 0;
      ++ltap;
      dz = ltap / 9 - 1;
      dy = (ltap / 3) % 3 - 1;
      dx = ltap % 3 - 1;
      forbid = 64 | (dz < 0) | (dz > 0) << 1 | (dy < 0) << 2 | (dy > 0) << 3 | (dx < 0) << 4 | (dx > 0) << 5;
      off0 = (dz * a.g.H + dy) * a.g.W + dx;
    }
    const int cb = lch * kBK;
    bf16 *as = As + buf * AE;
#pragma unroll
    for (int i = 0; i < RPT; ++i) {
      const int row = (tid >> 2) + i * (NTH / 4);
      const bool ok = (rm[i] & forbid) == 0;
      const bf16 *src;
      if (cb < a.c1) {
        // nearest upsampling: the neighbour's half-size cell moves by
        // floor((parity + d) / 2) along each axis
        const int oz = (((rm[i] >> 8) & 1) + dz) >> 1, oy = (((rm[i] >> 9) & 1) + dy) >> 1,
                  ox = (((rm[i] >> 10) & 1) + dx) >> 1;
        const int n = ok ? li[i] + (oz * H2 + oy) * W2 + ox : 0;
        src = a.x1 + (size_t)(unsigned)n * a.c1 + cb;
      } else {
        const int n = ok ? vi[i] + off0 : 0;
        src = a.x0 + (size_t)(unsigned)n * a.c0 + (cb - a.c1);
      }
      cp_async16(as + row * kAS + q * 8, ok ? src + q * 8 : a.w, ok ? 16 : 0);
    }
    bf16 *bs = Bs + buf * BE;
    const bf16 *wt = a.w + (size_t)ltap * cin + cb;
    for (int e = tid; e < BN * 4; e += NTH) {
      const int r = e >> 2, qq = e & 3;
      cp_async16(bs + r * kAS + qq * 8, wt + (size_t)(n0 + r) * 27 * cin + qq * 8, 16);
    }
    ++lch;
  };

  float acc[2][4][4];
#pragma unroll
  for (int i = 0; i < 2; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    if (st < ksteps) load(st);
    cp_async_commit();
  }
  for (int ks = 0; ks < ksteps; ++ks) {
    cp_async_wait1();  // kStages - 2 groups may stay in flight
    __syncthreads();
    if (ks + kStages - 1 < ksteps) load((ks + kStages - 1) % kStages);
    cp_async_commit();
    const bf16 *as = As + (ks % kStages) * AE, *bs = Bs + (ks % kStages) * BE;
#pragma unroll
    for (int kk = 0; kk < kBK; kk += 16) {
      uint32_t af[2][4], bfr[2][4];
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
        ldsm_x4(af[mi], as + (wm * 32 + mi * 16 + (lane & 15)) * kAS + kk + (lane >> 4) * 8);
#pragma unroll
      for (int nj2 = 0; nj2 < 2; ++nj2)
        ldsm_x4(bfr[nj2], bs + (wn * 32 + nj2 * 16 + ((lane >> 4) << 3) + (lane & 7)) * kAS + kk +
                              ((lane >> 3) & 1) * 8);
#pragma unroll
      for (int mi = 0; mi < 2; ++mi)
#pragma unroll
        for (int nj2 = 0; nj2 < 2; ++nj2) {
          mma_bf16(acc[mi][2 * nj2], af[mi], bfr[nj2][0], bfr[nj2][1]);
          mma_bf16(acc[mi][2 * nj2 + 1], af[mi], bfr[nj2][2], bfr[nj2][3]);
        }
    }
  }

  const int gq = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int mi = 0; mi < 2; ++mi)
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const int row = m0 + wm * 32 + mi * 16 + gq + 8 * h;
      if (row >= V) continue;
#pragma unroll
      for (int nj = 0; nj < 4; ++nj) {
        const int col = n0 + wn * 32 + nj * 8 + 2 * t4;
        float v0 = acc[mi][nj][2 * h], v1 = acc[mi][nj][2 * h + 1];
        if (a.bias) {
          v0 += a.bias[col];
          v1 += a.bias[col + 1];
        }
        if (a.relu) {
          v0 = fmaxf(v0, 0.f);
          v1 = fmaxf(v1, 0.f);
        }
        const size_t o = (size_t)row * a.cout + col;
        if (a.mask) {
          const __nv_bfloat162 m = *reinterpret_cast<const __nv_bfloat162 *>(a.mask + o);
          v0 = __bfloat162float(m.x) > 0.f ? v0 : 0.f;
          v1 = __bfloat162float(m.y) > 0.f ? v1 : 0.f;
        }
        *reinterpret_cast<__nv_bfloat162 *>(a.y + o) = __floats2bfloat162_rn(v0, v1);
      }
    }
}

// ---------------------------------------------------------------- weight gradient
struct WgradArgs {
  const bf16 *g;    // [V][cout] output gradient (ReLU mask applied)
  const bf16 *x0;
  const bf16 *x1;
  float *dw;        // [cout][27][c1 + c0], accumulated
  int c0, c1, cout, chunk;
  int first;        // 1: x0 holds the first layer's 27 neighbour values per voxel (+5 zeros); one
                    // unshifted "tap", output dw[o][j] for j < 27
  Vol vol;
};

constexpr int kWS = 64;  // voxels per weight-gradient stage

template <int MT>
constexpr int wgrad_smem_bytes() {
  return kStages * kWS * ((MT + 8) + kAS) * (int)sizeof(bf16);
}

// CTA: MT output channels x 32 input channels of one tap, over one chunk of
// voxels in stages of kWS; four warps, each (MT / 2) x 16.
template <int MT>
__global__ void __launch_bounds__(128) conv_wgrad_kernel(WgradArgs a) {
  constexpr int GS = MT + 8;  // shared row stride of the gradient tile (bf16)
  constexpr int GE = kWS * GS, XE = kWS * kAS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16 *Gs = reinterpret_cast<bf16 *>(smem_raw);
  bf16 *Xs = Gs + kStages * GE;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int wm = warp & 1, wn = warp >> 1;
  const int cin = a.c0 + a.c1, nch = cin / kBK;
  const int tap = a.first ? 13 : blockIdx.x / nch, cb = (blockIdx.x - (a.first ? 0 : tap) * nch) * kBK;
  const int dz = tap / 9 - 1, dy = (tap / 3) % 3 - 1, dx = tap % 3 - 1;
  const int co0 = blockIdx.y * MT;
  const Vol &g = a.vol;
  const int V = nvox(g);
  const int pbeg = blockIdx.z * a.chunk, pend = min(V, pbeg + a.chunk);
  if (pbeg >= pend) return;
  const int nst = (pend - pbeg + kWS - 1) / kWS;
  const int off0 = (dz * g.H + dy) * g.W + dx;
  const int D2 = g.D >> 1, H2 = g.H >> 1, W2 = g.W >> 1;

  // the two X rows this thread gathers (r0, r0 + 32), advanced by kWS per stage
  const int r0 = tid >> 2, xq = tid & 3;
  int vb[2], vz[2], vy[2], vx[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) decode(min(pbeg + r0 + 32 * i, V - 1), g, vb[i], vz[i], vy[i], vx[i]);
  auto load = [&](int st, int buf) {
    const int pb = pbeg + st * kWS;
    bf16 *gs = Gs + buf * GE;
#pragma unroll
    for (int i = 0; i < MT / 16; ++i) {
      const int e = tid + 128 * i;
      const int r = e / (MT / 8), qq = e % (MT / 8);
      const int p = pb + r;
      const bool ok = p < pend;
      cp_async16(gs + r * GS + qq * 8, ok ? a.g + (size_t)p * a.cout + co0 + qq * 8 : a.g, ok ? 16 : 0);
    }
    bf16 *xs = Xs + buf * XE;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = r0 + 32 * i, p = pb + r;
      const int z = vz[i] + dz, y = vy[i] + dy, x = vx[i] + dx;
      const bool ok = p < pend && z >= 0 && z < g.D && y >= 0 && y < g.H && x >= 0 && x < g.W;
      const bf16 *src = a.g;
      if (ok) {
        if (cb < a.c1)
          src = a.x1 + (size_t)(unsigned)(((vb[i] * D2 + (z >> 1)) * H2 + (y >> 1)) * W2 + (x >> 1)) * a.c1 + cb +
                xq * 8;
        else
          src = a.x0 + (size_t)(unsigned)(p + off0) * a.c0 + (cb - a.c1) + xq * 8;
      }
      cp_async16(xs + r * kAS + xq * 8, src, ok ? 16 : 0);
      vx[i] += kWS;
      while (vx[i] >= g.W) {
        vx[i] -= g.W;
        if (++vy[i] == g.H) {
          vy[i] = 0;
          if (++vz[i] == g.D) {
            vz[i] = 0;
            ++vb[i];
          }
        }
      }
    }
  };

  constexpr int MI = MT / 32;  // m16 tiles per warp (the warp owns MT / 2 rows)
  float acc[MI][2][4];
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < 2; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    if (st < nst) load(st, st);
    cp_async_commit();
  }
  const int mat = lane >> 3, r8 = lane & 7;
  for (int st = 0; st < nst; ++st) {
    cp_async_wait1();
    __syncthreads();
    if (st + kStages - 1 < nst) load(st + kStages - 1, (st + kStages - 1) % kStages);
    cp_async_commit();
    const bf16 *gs = Gs + (st % kStages) * GE, *xs = Xs + (st % kStages) * XE;
#pragma unroll
    for (int kk = 0; kk < kWS; kk += 16) {
      uint32_t bfr[4];  // B[k = voxel][n = channel] from Xs[k][n], transposed on load
      ldsm_x4_t(bfr, xs + (kk + (mat & 1) * 8 + r8) * kAS + wn * 16 + (mat >> 1) * 8);
#pragma unroll
      for (int mi = 0; mi < MI; ++mi) {
        uint32_t af[4];  // A[m = out channel][k = voxel] from Gs[k][m], transposed on load
        ldsm_x4_t(af, gs + (kk + (mat >> 1) * 8 + r8) * GS + wm * (MT / 2) + mi * 16 + (mat & 1) * 8);
        mma_bf16(acc[mi][0], af, bfr[0], bfr[1]);
        mma_bf16(acc[mi][1], af, bfr[2], bfr[3]);
      }
    }
  }

  const int gq = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int nj = 0; nj < 2; ++nj)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int o = co0 + wm * (MT / 2) + mi * 16 + gq + 8 * (e >> 1);
        const int c = cb + wn * 16 + nj * 8 + 2 * t4 + (e & 1);
        if (a.first) {
          if (c < 27) atomicAdd(a.dw + o * 27 + c, acc[mi][nj][e]);
        } else {
          atomicAdd(a.dw + ((size_t)o * 27 + tap) * cin + c, acc[mi][nj][e]);
        }
      }
}

template <int MT>
constexpr int wgrad4_smem_bytes() {
  return kStages * kWS * ((MT + 8) + 4 * kAS) * (int)sizeof(bf16);
}

// Four taps per CTA: warp w owns tap 4 t + w (t = blockIdx.x / nch) for all MT
// output channels x 32 input channels, so the gradient tile of a stage is
// shared by four warps and each warp runs (MT / 16) x 4 fragments per 16 voxels.
template <int MT>
__global__ void __launch_bounds__(128) conv_wgrad4_kernel(WgradArgs a) {
  constexpr int GS = MT + 8;
  constexpr int GE = kWS * GS, XE = kWS * kAS;
  extern __shared__ __align__(16) unsigned char smem_raw[];
  bf16 *Gs = reinterpret_cast<bf16 *>(smem_raw);
  bf16 *Xs = Gs + kStages * GE;  // [stage][tap][voxel][channel]
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int cin = a.c0 + a.c1, nch = cin / kBK;
  const int tg = blockIdx.x / nch, cb = (blockIdx.x - tg * nch) * kBK;
  const int co0 = blockIdx.y * MT;
  const Vol &g = a.vol;
  const int V = nvox(g);
  const int pbeg = blockIdx.z * a.chunk, pend = min(V, pbeg + a.chunk);
  if (pbeg >= pend) return;
  const int nst = (pend - pbeg + kWS - 1) / kWS;
  const int D2 = g.D >> 1, H2 = g.H >> 1, W2 = g.W >> 1;
  int tdz[4], tdy[4], tdx[4], toff[4];
  bool tv[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int t = 4 * tg + j;
    tv[j] = t < 27;
    tdz[j] = t / 9 - 1;
    tdy[j] = (t / 3) % 3 - 1;
    tdx[j] = t % 3 - 1;
    toff[j] = (tdz[j] * g.H + tdy[j]) * g.W + tdx[j];
  }

  const int r0 = tid >> 2, xq = tid & 3;
  int vb[2], vz[2], vy[2], vx[2];
#pragma unroll
  for (int i = 0; i < 2; ++i) decode(min(pbeg + r0 + 32 * i, V - 1), g, vb[i], vz[i], vy[i], vx[i]);
  auto load = [&](int st, int buf) {
    const int pb = pbeg + st * kWS;
    bf16 *gs = Gs + buf * GE;
#pragma unroll
    for (int i = 0; i < MT / 16; ++i) {
      const int e = tid + 128 * i;
      const int r = e / (MT / 8), qq = e % (MT / 8);
      const int p = pb + r;
      const bool ok = p < pend;
      cp_async16(gs + r * GS + qq * 8, ok ? a.g + (size_t)p * a.cout + co0 + qq * 8 : a.g, ok ? 16 : 0);
    }
    bf16 *xs = Xs + buf * 4 * XE;
#pragma unroll
    for (int i = 0; i < 2; ++i) {
      const int r = r0 + 32 * i, p = pb + r;
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const int z = vz[i] + tdz[j], y = vy[i] + tdy[j], x = vx[i] + tdx[j];
        const bool ok = tv[j] && p < pend && z >= 0 && z < g.D && y >= 0 && y < g.H && x >= 0 && x < g.W;
        const bf16 *src = a.g;
        if (ok) {
          if (cb < a.c1)
            src = a.x1 + (size_t)(unsigned)(((vb[i] * D2 + (z >> 1)) * H2 + (y >> 1)) * W2 + (x >> 1)) * a.c1 + cb +
                  xq * 8;
          else
            src = a.x0 + (size_t)(unsigned)(p + toff[j]) * a.c0 + (cb - a.c1) + xq * 8;
        }
        cp_async16(xs + j * XE + r * kAS + xq * 8, src, ok ? 16 : 0);
      }
      vx[i] += kWS;
      while (vx[i] >= g.W) {
        vx[i] -= g.W;
        if (++vy[i] == g.H) {
          vy[i] = 0;
          if (++vz[i] == g.D) {
            vz[i] = 0;
            ++vb[i];
          }
        }
      }
    }
  };

  constexpr int MI = MT / 16;
  float acc[MI][4][4];
#pragma unroll
  for (int i = 0; i < MI; ++i)
#pragma unroll
    for (int j = 0; j < 4; ++j)
#pragma unroll
      for (int e = 0; e < 4; ++e) acc[i][j][e] = 0.f;

#pragma unroll
  for (int st = 0; st < kStages - 1; ++st) {
    if (st < nst) load(st, st);
    cp_async_commit();
  }
  const int mat = lane >> 3, r8 = lane & 7;
  const bool active = 4 * tg + warp < 27;
  for (int st = 0; st < nst; ++st) {
    cp_async_wait1();
    __syncthreads();
    if (st + kStages - 1 < nst) load(st + kStages - 1, (st + kStages - 1) % kStages);
    cp_async_commit();
    if (!active) continue;
    const bf16 *gs = Gs + (st % kStages) * GE, *xs = Xs + ((st % kStages) * 4 + warp) * XE;
#pragma unroll
    for (int kk = 0; kk < kWS; kk += 16) {
      uint32_t bfr[2][4];
#pragma unroll
      for (int nj2 = 0; nj2 < 2; ++nj2)
        ldsm_x4_t(bfr[nj2], xs + (kk + (mat & 1) * 8 + r8) * kAS + nj2 * 16 + (mat >> 1) * 8);
#pragma unroll
      for (int mi = 0; mi < MI; ++mi) {
        uint32_t af[4];
        ldsm_x4_t(af, gs + (kk + (mat >> 1) * 8 + r8) * GS + mi * 16 + (mat & 1) * 8);
#pragma unroll
        for (int nj2 = 0; nj2 < 2; ++nj2) {
          mma_bf16(acc[mi][2 * nj2], af, bfr[nj2][0], bfr[nj2][1]);
          mma_bf16(acc[mi][2 * nj2 + 1], af, bfr[nj2][2], bfr[nj2][3]);
        }
      }
    }
  }
  if (!active) return;
  const int tap = 4 * tg + warp;
  const int gq = lane >> 2, t4 = lane & 3;
#pragma unroll
  for (int mi = 0; mi < MI; ++mi)
#pragma unroll
    for (int nj = 0; nj < 4; ++nj)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int o = co0 + mi * 16 + gq + 8 * (e >> 1);
        const int c = cb + nj * 8 + 2 * t4 + (e & 1);
        atomicAdd(a.dw + ((size_t)o * 27 + tap) * cin + c, acc[mi][nj][e]);
      }
}

// ---------------------------------------------------------------- first layer (one input channel)
__global__ void __launch_bounds__(256) conv_first_kernel(const float *v, const bf16 *w, const float *bias, bf16 *y,
                                                         Vol g) {
  __shared__ float ws[32 * 27];
  __shared__ float bs[32];
  for (int i = threadIdx.x; i < 32 * 27; i += blockDim.x) ws[i] = __bfloat162float(w[i]);
  if (threadIdx.x < 32) bs[threadIdx.x] = bias[threadIdx.x];
  __syncthreads();
  const int V = nvox(g);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < V; p += gridDim.x * blockDim.x) {
    int b, z, yy, x;
    decode(p, g, b, z, yy, x);
    float nb[27];
#pragma unroll
    for (int t = 0; t < 27; ++t) {
      const int zz = z + t / 9 - 1, y2 = yy + (t / 3) % 3 - 1, x2 = x + t % 3 - 1;
      const bool ok = zz >= 0 && zz < g.D && y2 >= 0 && y2 < g.H && x2 >= 0 && x2 < g.W;
      nb[t] = ok ? v[(((size_t)b * g.D + zz) * g.H + y2) * g.W + x2] : 0.f;
    }
    uint4 out[4];
    uint32_t *o32 = reinterpret_cast<uint32_t *>(out);
#pragma unroll
    for (int c = 0; c < 32; c += 2) {
      float s0 = bs[c], s1 = bs[c + 1];
#pragma unroll
      for (int t = 0; t < 27; ++t) {
        s0 = fmaf(ws[c * 27 + t], nb[t], s0);
        s1 = fmaf(ws[(c + 1) * 27 + t], nb[t], s1);
      }
      __nv_bfloat162 h = __floats2bfloat162_rn(fmaxf(s0, 0.f), fmaxf(s1, 0.f));
      o32[c / 2] = *reinterpret_cast<uint32_t *>(&h);
    }
    uint4 *dst = reinterpret_cast<uint4 *>(y + (size_t)p * 32);
#pragma unroll
    for (int i = 0; i < 4; ++i) dst[i] = out[i];
  }
}

// col[p][j] = v[p + delta_j] for the 27 taps j (zero outside the volume), then
// five zeros: the first layer's input as 32 BF16 channels, so its weight
// gradient runs on the tensor-core weight-gradient kernel.
__global__ void __launch_bounds__(256) im2col_first_kernel(const float *v, bf16 *col, Vol g) {
  const int V = nvox(g);
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < V; p += gridDim.x * blockDim.x) {
    int b, z, y, x;
    decode(p, g, b, z, y, x);
    float nb[32];
#pragma unroll
    for (int t = 0; t < 32; ++t) {
      nb[t] = 0.f;
      if (t < 27) {
        const int zz = z + t / 9 - 1, y2 = y + (t / 3) % 3 - 1, x2 = x + t % 3 - 1;
        if (zz >= 0 && zz < g.D && y2 >= 0 && y2 < g.H && x2 >= 0 && x2 < g.W)
          nb[t] = v[(((size_t)b * g.D + zz) * g.H + y2) * g.W + x2];
      }
    }
#pragma unroll
    for (int c8 = 0; c8 < 4; ++c8) store8(col + (size_t)p * 32 + c8 * 8, nb + 8 * c8);
  }
}

// ---------------------------------------------------------------- bias gradient
// out[c] += sum_p G[p][c] over one chunk of voxels (C divides 256).
__global__ void __launch_bounds__(256) colsum_kernel(const bf16 *G, int V, int C, int chunk, float *out) {
  __shared__ float red[256];
  const int c = threadIdx.x % C, r0 = threadIdx.x / C, R = 256 / C;
  const int pbeg = blockIdx.x * chunk, pend = min(V, pbeg + chunk);
  float s = 0.f;
  for (int p = pbeg + r0; p < pend; p += R) s += __bfloat162float(G[(size_t)p * C + c]);
  red[threadIdx.x] = s;
  __syncthreads();
  if (r0 == 0) {
    for (int r = 1; r < R; ++r) s += red[r * C + c];
    atomicAdd(out + c, s);
  }
}

// ---------------------------------------------------------------- pooling and its transposes
// mode 0: y[q] = mean of the 8 children of q in x (x: C channels).
// mode 1: y[q] = (sum of the 8 children of q in x[., coff : coff + C] (stride cx))
//         zeroed where mask[q] <= 0 (transpose of nearest upsampling, then ReLU mask).
__global__ void pool_kernel(const bf16 *x, int cx, int coff, const bf16 *mask, bf16 *y, int C, Vol lo, int mode) {
  const int pieces = C / 8;
  const long long n = (long long)nvox(lo) * pieces;
  const int Dh = 2 * lo.D, Hh = 2 * lo.H, Wh = 2 * lo.W;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < n; it += (long long)gridDim.x * blockDim.x) {
    const int q = (int)(it / pieces), pc = (int)(it % pieces);
    int b, z, yy, xx;
    decode(q, lo, b, z, yy, xx);
    float s[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      const size_t ch = (((size_t)b * Dh + 2 * z + (c >> 2)) * Hh + 2 * yy + ((c >> 1) & 1)) * Wh + 2 * xx + (c & 1);
      float f[8];
      load8(x + ch * cx + coff + pc * 8, f);
#pragma unroll
      for (int i = 0; i < 8; ++i) s[i] += f[i];
    }
    if (mode == 0) {
#pragma unroll
      for (int i = 0; i < 8; ++i) s[i] *= 0.125f;
    } else {
      float m[8];
      load8(mask + (size_t)q * C + pc * 8, m);
#pragma unroll
      for (int i = 0; i < 8; ++i) s[i] = m[i] > 0.f ? s[i] : 0.f;
    }
    store8(y + (size_t)q * C + pc * 8, s);
  }
}

// y[p] = (glo[parent(p)] / 8 + ghi[p, coff : coff + C]) zeroed where mask[p] <= 0:
// the gradient of a tensor that feeds both a pooling and a skip connection.
__global__ void combine_kernel(const bf16 *glo, const bf16 *ghi, int chi, int coff, const bf16 *mask, bf16 *y, int C,
                               Vol hi) {
  const int pieces = C / 8;
  const long long n = (long long)nvox(hi) * pieces;
  const int Dl = hi.D / 2, Hl = hi.H / 2, Wl = hi.W / 2;
  for (long long it = blockIdx.x * (long long)blockDim.x + threadIdx.x; it < n; it += (long long)gridDim.x * blockDim.x) {
    const int p = (int)(it / pieces), pc = (int)(it % pieces);
    int b, z, yy, xx;
    decode(p, hi, b, z, yy, xx);
    const size_t par = (((size_t)b * Dl + (z >> 1)) * Hl + (yy >> 1)) * Wl + (xx >> 1);
    float lo[8], h[8], m[8], s[8];
    load8(glo + par * C + pc * 8, lo);
    load8(ghi + (size_t)p * chi + coff + pc * 8, h);
    load8(mask + (size_t)p * C + pc * 8, m);
#pragma unroll
    for (int i = 0; i < 8; ++i) s[i] = m[i] > 0.f ? fmaf(0.125f, lo[i], h[i]) : 0.f;
    store8(y + (size_t)p * C + pc * 8, s);
  }
}

// ---------------------------------------------------------------- head
// h = Wh f + bh; u = v + h0, s = h1, t = h2.  hp: Wh[3][32] then bh[3] (FP32).
__global__ void __launch_bounds__(256) head_fwd_kernel(const bf16 *f, const float *v, const float *hp, float *u,
                                                       float *s, float *t, int V) {
  __shared__ float w[kHeadIn * kHeadOut + kHeadOut];
  for (int i = threadIdx.x; i < kHeadIn * kHeadOut + kHeadOut; i += blockDim.x) w[i] = hp[i];
  __syncthreads();
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < V; p += gridDim.x * blockDim.x) {
    float h0 = w[96], h1 = w[97], h2 = w[98];
#pragma unroll
    for (int c8 = 0; c8 < 4; ++c8) {
      float fv[8];
      load8(f + (size_t)p * 32 + c8 * 8, fv);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int c = c8 * 8 + i;
        h0 = fmaf(w[c], fv[i], h0);
        h1 = fmaf(w[32 + c], fv[i], h1);
        h2 = fmaf(w[64 + c], fv[i], h2);
      }
    }
    u[p] = v[p] + h0;
    s[p] = h1;
    t[p] = h2;
  }
}

// Loss, head gradients and the gradient into d1b.  With e_j = pred_j - target_j
// and n = 3 V: loss += sum e_j^2 / n; dh_j = 2 e_j / n; dWh[j][c] += dh_j f[c];
// dbh[j] += dh_j; G[p][c] = (sum_j dh_j Wh[j][c]) where f[c] > 0.
__global__ void __launch_bounds__(256) head_bwd_kernel(const bf16 *f, const float *v, const float *hp,
                                                       const float *tu, const float *ts, const float *tt, int V,
                                                       float inv_n, bf16 *G, float *dwh, double *loss) {
  __shared__ float w[kHeadIn * kHeadOut + kHeadOut];
  __shared__ float red[8][kHeadIn * kHeadOut + kHeadOut];
  __shared__ double lred[8];
  for (int i = threadIdx.x; i < kHeadIn * kHeadOut + kHeadOut; i += blockDim.x) w[i] = hp[i];
  __syncthreads();
  float gw[kHeadOut][kHeadIn];
  float gb[kHeadOut] = {0.f, 0.f, 0.f};
#pragma unroll
  for (int j = 0; j < kHeadOut; ++j)
#pragma unroll
    for (int c = 0; c < kHeadIn; ++c) gw[j][c] = 0.f;
  double lsum = 0.0;
  for (int p = blockIdx.x * blockDim.x + threadIdx.x; p < V; p += gridDim.x * blockDim.x) {
    float fv[32];
#pragma unroll
    for (int c8 = 0; c8 < 4; ++c8) load8(f + (size_t)p * 32 + c8 * 8, fv + 8 * c8);
    float h0 = w[96], h1 = w[97], h2 = w[98];
#pragma unroll
    for (int c = 0; c < 32; ++c) {
      h0 = fmaf(w[c], fv[c], h0);
      h1 = fmaf(w[32 + c], fv[c], h1);
      h2 = fmaf(w[64 + c], fv[c], h2);
    }
    const float e0 = (v[p] + h0) - tu[p], e1 = h1 - ts[p], e2 = h2 - tt[p];
    lsum += (double)e0 * e0 + (double)e1 * e1 + (double)e2 * e2;
    const float d0 = 2.f * e0 * inv_n, d1 = 2.f * e1 * inv_n, d2 = 2.f * e2 * inv_n;
    gb[0] += d0;
    gb[1] += d1;
    gb[2] += d2;
#pragma unroll
    for (int c8 = 0; c8 < 4; ++c8) {
      float go[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const int c = c8 * 8 + i;
        gw[0][c] = fmaf(d0, fv[c], gw[0][c]);
        gw[1][c] = fmaf(d1, fv[c], gw[1][c]);
        gw[2][c] = fmaf(d2, fv[c], gw[2][c]);
        const float gc = fmaf(d0, w[c], fmaf(d1, w[32 + c], d2 * w[64 + c]));
        go[i] = fv[c] > 0.f ? gc : 0.f;
      }
      store8(G + (size_t)p * 32 + c8 * 8, go);
    }
  }
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int j = 0; j < kHeadOut; ++j)
#pragma unroll
    for (int c = 0; c < kHeadIn; ++c) {
      float x = gw[j][c];
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
      if (lane == 0) red[warp][j * kHeadIn + c] = x;
    }
#pragma unroll
  for (int j = 0; j < kHeadOut; ++j) {
    float x = gb[j];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) x += __shfl_xor_sync(0xffffffffu, x, o);
    if (lane == 0) red[warp][96 + j] = x;
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) lsum += __shfl_xor_sync(0xffffffffu, lsum, o);
  if (lane == 0) lred[warp] = lsum;
  __syncthreads();
  if (threadIdx.x < kHeadIn * kHeadOut + kHeadOut) {
    float x = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) x += red[i][threadIdx.x];
    atomicAdd(dwh + threadIdx.x, x);
  }
  if (threadIdx.x == 0) {
    double x = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) x += lred[i];
    atomicAdd(loss, x * (double)inv_n);
  }
}

// ---------------------------------------------------------------- optimiser and weight packing
__global__ void adam_kernel(float *theta, const float *g, float *m, float *s, long long n, float lr, float b1,
                            float b2, float eps, float c1, float c2) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x) {
    const float gi = g[i];
    const float mi = fmaf(b1, m[i], (1.f - b1) * gi);
    const float si = fmaf(b2, s[i], (1.f - b2) * gi * gi);
    m[i] = mi;
    s[i] = si;
    theta[i] -= lr * (mi * c1) / (sqrtf(si * c2) + eps);
  }
}

// BF16 copies of the weights: wf in the training layout [o][tap][c], wb as
// wb[c][26 - tap][o] (the input-gradient conv), hp = the head with its weights
// rounded to BF16 and its bias in FP32.
__global__ void pack_kernel(const float *theta, LayerTable t, bf16 *wf, bf16 *wb, float *hp) {
  for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < t.total; i += (long long)gridDim.x * blockDim.x) {
    const float x = theta[i];
    if (i >= t.hw_off) {
      const long long j = i - t.hw_off;
      hp[j] = i < t.hb_off ? __bfloat162float(__float2bfloat16_rn(x)) : x;
      continue;
    }
    int l = 0;
    while (l + 1 < kLayers && i >= t.woff[l + 1]) ++l;
    if (i >= t.boff[l]) continue;  // biases stay FP32 in theta
    const long long loc = i - t.woff[l];
    const int ci = t.cin[l], co = t.cout[l];
    const int o = (int)(loc / (27LL * ci));
    const int rem = (int)(loc - (long long)o * 27 * ci);
    const int tap = rem / ci, c = rem - tap * ci;
    const bf16 h = __float2bfloat16_rn(x);
    wf[i] = h;
    wb[t.woff[l] + ((long long)c * 27 + (26 - tap)) * co + o] = h;
  }
}

}  // namespace

// ====================================================================== host side
struct s3ttv_net {
  int device = 0, num_sms = 1;
  cudaStream_t stream = nullptr;
  bool own_stream = false;
  char err[256] = {0};
  LayerTable tab;
  float *theta = nullptr, *grad = nullptr, *m1 = nullptr, *m2 = nullptr, *hp = nullptr;
  bf16 *wf = nullptr, *wb = nullptr;
  double *loss = nullptr;
  long long adam_t = 0;
  bool have_params = false;
  // shape-dependent workspace
  Vol vol = {0, 0, 0, 0};
  void *arena = nullptr;
  size_t arena_bytes = 0;
  float *stage = nullptr;
  size_t stage_floats = 0;
  bf16 *e1a, *e1b, *d1a, *d1b, *gA0, *gB0, *gC0;
  bf16 *p1, *e2a, *e2b, *d2a, *d2b, *gA1, *gB1, *gC1;
  bf16 *p2, *ba, *bb, *gB2, *gC2;
};

namespace {

int nfail(s3ttv_net *n, int status, const char *fmt, ...) {
  if (n) {
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(n->err, sizeof(n->err), fmt, ap);
    va_end(ap);
  }
  return status;
}

#define NCU(call)                                                                           \
  do {                                                                                      \
    cudaError_t e_ = (call);                                                                \
    if (e_ != cudaSuccess)                                                                  \
      return nfail(net, S3TTV_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_));       \
  } while (0)

struct Guard {
  int prev = -1;
  explicit Guard(int dev) {
    if (cudaGetDevice(&prev) != cudaSuccess) prev = -1;
    cudaSetDevice(dev);
  }
  ~Guard() {
    if (prev >= 0) cudaSetDevice(prev);
  }
};

bool on_device(const void *p) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, p) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  return at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
}

int grid_for(const s3ttv_net *net, long long items, int threads) {
  long long g = (items + threads - 1) / threads;
  const long long cap = (long long)net->num_sms * 8;
  if (g > cap) g = cap;
  return g < 1 ? 1 : (int)g;
}

cudaError_t launch_conv(const s3ttv_net *net, const bf16 *x0, int c0, const bf16 *x1, int c1, const bf16 *w,
                        const float *bias, const bf16 *mask, bf16 *y, int cout, bool relu, Vol g) {
  ConvArgs a{x0, x1, w, bias, mask, y, c0, c1, cout, relu ? 1 : 0, g};
  const int V = nvox(g);
  if (cout % 64 == 0) {
    dim3 grid((V + 127) / 128, cout / 64);
    conv_fwd_kernel<128, 64><<<grid, 256, conv_smem_bytes<128, 64>(), net->stream>>>(a);
  } else {
    dim3 grid((V + 255) / 256, cout / 32);
    conv_fwd_kernel<256, 32><<<grid, 256, conv_smem_bytes<256, 32>(), net->stream>>>(a);
  }
  return cudaGetLastError();
}

cudaError_t launch_wgrad(const s3ttv_net *net, const bf16 *G, int cout, const bf16 *x0, int c0, const bf16 *x1,
                         int c1, float *dw, Vol g) {
  const int V = nvox(g);
  // up to 64 output channels: four taps per CTA; 128: one tap per CTA
  const bool four = cout <= 64;
  const int MT = four ? cout : 128;
  const int gx = (four ? 7 : 27) * ((c0 + c1) / kBK), gy = cout / MT;
  const long long target = (long long)net->num_sms * 8;
  long long z = (target + (long long)gx * gy - 1) / ((long long)gx * gy);
  const long long zmax = (V + 511) / 512;
  if (z > zmax) z = zmax;
  if (z < 1) z = 1;
  int chunk = (int)(((V + z - 1) / z + kWS - 1) / kWS * kWS);
  z = (V + chunk - 1) / chunk;
  WgradArgs a{G, x0, x1, dw, c0, c1, cout, chunk, 0, g};
  dim3 grid(gx, gy, (unsigned)z);
  if (MT == 128)
    conv_wgrad_kernel<128><<<grid, 128, wgrad_smem_bytes<128>(), net->stream>>>(a);
  else if (MT == 64)
    conv_wgrad4_kernel<64><<<grid, 128, wgrad4_smem_bytes<64>(), net->stream>>>(a);
  else
    conv_wgrad4_kernel<32><<<grid, 128, wgrad4_smem_bytes<32>(), net->stream>>>(a);
  return cudaGetLastError();
}

cudaError_t launch_colsum(const s3ttv_net *net, const bf16 *G, int V, int C, float *out) {
  const int blocks = grid_for(net, V, 256);
  const int chunk = (V + blocks - 1) / blocks;
  colsum_kernel<<<(V + chunk - 1) / chunk, 256, 0, net->stream>>>(G, V, C, chunk, out);
  return cudaGetLastError();
}

Vol half(const Vol &g) { return Vol{g.B, g.D / 2, g.H / 2, g.W / 2}; }

int ensure_workspace(s3ttv_net *net, const Vol &g) {
  const size_t V0 = (size_t)nvox(g), V1 = V0 / 8, V2 = V0 / 64;
  // elements: level 0: 4 x 32 activations, gA0 96, gB0 / gC0 32;
  // level 1: p1 32, 4 x 64, gA1 192, gB1 / gC1 64; level 2: p2 64, 2 x 128, gB2 / gC2 128
  const size_t sz[] = {V0 * 32, V0 * 32, V0 * 32, V0 * 32, V0 * 96, V0 * 32, V0 * 32,
                       V1 * 32, V1 * 64, V1 * 64, V1 * 64, V1 * 64, V1 * 192, V1 * 64, V1 * 64,
                       V2 * 64, V2 * 128, V2 * 128, V2 * 128, V2 * 128};
  bf16 **dst[] = {&net->e1a, &net->e1b, &net->d1a, &net->d1b, &net->gA0, &net->gB0, &net->gC0,
                  &net->p1, &net->e2a, &net->e2b, &net->d2a, &net->d2b, &net->gA1, &net->gB1, &net->gC1,
                  &net->p2, &net->ba, &net->bb, &net->gB2, &net->gC2};
  size_t total = 0;
  for (size_t e : sz) total += (e * sizeof(bf16) + 255) / 256 * 256;
  if (total > net->arena_bytes) {
    if (net->arena) cudaFree(net->arena);
    net->arena = nullptr;
    net->arena_bytes = 0;
    if (cudaMalloc(&net->arena, total) != cudaSuccess) {
      cudaGetLastError();
      return nfail(net, S3TTV_ENOMEM, "workspace of %zu bytes", total);
    }
    net->arena_bytes = total;
  }
  char *p = (char *)net->arena;
  for (size_t i = 0; i < sizeof(sz) / sizeof(sz[0]); ++i) {
    *dst[i] = (bf16 *)p;
    p += (sz[i] * sizeof(bf16) + 255) / 256 * 256;
  }
  net->vol = g;
  return S3TTV_OK;
}

int ensure_stage(s3ttv_net *net, size_t floats) {
  if (floats <= net->stage_floats) return S3TTV_OK;
  if (net->stage) cudaFree(net->stage);
  net->stage = nullptr;
  net->stage_floats = 0;
  if (cudaMalloc(&net->stage, floats * sizeof(float)) != cudaSuccess) {
    cudaGetLastError();
    return nfail(net, S3TTV_ENOMEM, "staging buffer of %zu floats", floats);
  }
  net->stage_floats = floats;
  return S3TTV_OK;
}

int check_shape(s3ttv_net *net, int B, int D, int H, int W) {
  if (!net) return S3TTV_EINVAL;
  if (B < 1 || D < 4 || H < 4 || W < 4 || D % 4 || H % 4 || W % 4)
    return nfail(net, S3TTV_EINVAL, "need B >= 1 and D, H, W positive multiples of 4 (got %d %d %d %d)", B, D, H, W);
  if ((long long)B * D * H * W > kMaxVoxels)
    return nfail(net, S3TTV_EUNSUPPORTED, "B*D*H*W above %lld voxels", kMaxVoxels);
  if (!net->have_params) return nfail(net, S3TTV_ESTATE, "parameters not set (s3ttv_net_set_params)");
  return S3TTV_OK;
}

// Device copies of the host inputs: slot i of the stage holds input i.
int stage_inputs(s3ttv_net *net, const float **ptrs, int count, size_t n, const float **dev) {
  int need = 0;
  for (int i = 0; i < count; ++i) need += on_device(ptrs[i]) ? 0 : 1;
  if (need) {
    int rc = ensure_stage(net, (size_t)(count + 3) * n);
    if (rc) return rc;
  }
  for (int i = 0; i < count; ++i) {
    if (on_device(ptrs[i])) {
      dev[i] = ptrs[i];
    } else {
      float *d = net->stage + (size_t)i * n;
      NCU(cudaMemcpyAsync(d, ptrs[i], n * sizeof(float), cudaMemcpyHostToDevice, net->stream));
      dev[i] = d;
    }
  }
  return S3TTV_OK;
}

const bf16 *wf(const s3ttv_net *net, int l) { return net->wf + net->tab.woff[l]; }
const bf16 *wbk(const s3ttv_net *net, int l) { return net->wb + net->tab.woff[l]; }
const float *bias(const s3ttv_net *net, int l) { return net->theta + net->tab.boff[l]; }

int run_forward(s3ttv_net *net, const float *v, const Vol &g0) {
  const Vol g1 = half(g0), g2 = half(g1);
  const int V0 = nvox(g0), V1 = nvox(g1), V2 = nvox(g2);
  conv_first_kernel<<<grid_for(net, V0, 256), 256, 0, net->stream>>>(v, wf(net, 0), bias(net, 0), net->e1a, g0);
  NCU(cudaGetLastError());
  NCU(launch_conv(net, net->e1a, 32, nullptr, 0, wf(net, 1), bias(net, 1), nullptr, net->e1b, 32, true, g0));
  pool_kernel<<<grid_for(net, (long long)V1 * 4, 256), 256, 0, net->stream>>>(net->e1b, 32, 0, nullptr, net->p1, 32,
                                                                               g1, 0);
  NCU(cudaGetLastError());
  NCU(launch_conv(net, net->p1, 32, nullptr, 0, wf(net, 2), bias(net, 2), nullptr, net->e2a, 64, true, g1));
  NCU(launch_conv(net, net->e2a, 64, nullptr, 0, wf(net, 3), bias(net, 3), nullptr, net->e2b, 64, true, g1));
  pool_kernel<<<grid_for(net, (long long)V2 * 8, 256), 256, 0, net->stream>>>(net->e2b, 64, 0, nullptr, net->p2, 64,
                                                                               g2, 0);
  NCU(cudaGetLastError());
  NCU(launch_conv(net, net->p2, 64, nullptr, 0, wf(net, 4), bias(net, 4), nullptr, net->ba, 128, true, g2));
  NCU(launch_conv(net, net->ba, 128, nullptr, 0, wf(net, 5), bias(net, 5), nullptr, net->bb, 128, true, g2));
  NCU(launch_conv(net, net->e2b, 64, net->bb, 128, wf(net, 6), bias(net, 6), nullptr, net->d2a, 64, true, g1));
  NCU(launch_conv(net, net->d2a, 64, nullptr, 0, wf(net, 7), bias(net, 7), nullptr, net->d2b, 64, true, g1));
  NCU(launch_conv(net, net->e1b, 32, net->d2b, 64, wf(net, 8), bias(net, 8), nullptr, net->d1a, 32, true, g0));
  NCU(launch_conv(net, net->d1a, 32, nullptr, 0, wf(net, 9), bias(net, 9), nullptr, net->d1b, 32, true, g0));
  return S3TTV_OK;
}

// Gradient of the loss into net->grad (zeroed here) and the loss into net->loss.
int run_backward(s3ttv_net *net, const float *v, const float *tu, const float *ts, const float *tt, const Vol &g0) {
  const Vol g1 = half(g0), g2 = half(g1);
  const int V0 = nvox(g0), V1 = nvox(g1), V2 = nvox(g2);
  const LayerTable &T = net->tab;
  float *G = net->grad;
  NCU(cudaMemsetAsync(G, 0, sizeof(float) * T.total, net->stream));
  NCU(cudaMemsetAsync(net->loss, 0, sizeof(double), net->stream));
  const float inv_n = (float)(1.0 / (3.0 * (double)V0));
  head_bwd_kernel<<<grid_for(net, V0, 256), 256, 0, net->stream>>>(net->d1b, v, net->hp, tu, ts, tt, V0, inv_n,
                                                                   net->gB0, G + T.hw_off, net->loss);
  NCU(cudaGetLastError());
  auto wgrad = [&](int l, const bf16 *gout, const bf16 *x0, int c0, const bf16 *x1, int c1, const Vol &g) {
    cudaError_t e = launch_wgrad(net, gout, T.cout[l], x0, c0, x1, c1, G + T.woff[l], g);
    if (e == cudaSuccess) e = launch_colsum(net, gout, nvox(g), T.cout[l], G + T.boff[l]);
    return e;
  };
  // d1b: gB0 -> gC0 (masked by d1a)
  NCU(wgrad(9, net->gB0, net->d1a, 32, nullptr, 0, g0));
  NCU(launch_conv(net, net->gB0, 32, nullptr, 0, wbk(net, 9), nullptr, net->d1a, net->gC0, 32, false, g0));
  // d1a: gC0 -> gA0 [up(d2b) 64 | e1b 32]
  NCU(wgrad(8, net->gC0, net->e1b, 32, net->d2b, 64, g0));
  NCU(launch_conv(net, net->gC0, 32, nullptr, 0, wbk(net, 8), nullptr, nullptr, net->gA0, 96, false, g0));
  pool_kernel<<<grid_for(net, (long long)V1 * 8, 256), 256, 0, net->stream>>>(net->gA0, 96, 0, net->d2b, net->gB1,
                                                                               64, g1, 1);
  NCU(cudaGetLastError());
  // d2b: gB1 -> gC1 (masked by d2a)
  NCU(wgrad(7, net->gB1, net->d2a, 64, nullptr, 0, g1));
  NCU(launch_conv(net, net->gB1, 64, nullptr, 0, wbk(net, 7), nullptr, net->d2a, net->gC1, 64, false, g1));
  // d2a: gC1 -> gA1 [up(bb) 128 | e2b 64]
  NCU(wgrad(6, net->gC1, net->e2b, 64, net->bb, 128, g1));
  NCU(launch_conv(net, net->gC1, 64, nullptr, 0, wbk(net, 6), nullptr, nullptr, net->gA1, 192, false, g1));
  pool_kernel<<<grid_for(net, (long long)V2 * 16, 256), 256, 0, net->stream>>>(net->gA1, 192, 0, net->bb, net->gB2,
                                                                                128, g2, 1);
  NCU(cudaGetLastError());
  // bb: gB2 -> gC2 (masked by ba)
  NCU(wgrad(5, net->gB2, net->ba, 128, nullptr, 0, g2));
  NCU(launch_conv(net, net->gB2, 128, nullptr, 0, wbk(net, 5), nullptr, net->ba, net->gC2, 128, false, g2));
  // ba: gC2 -> gradient of p2 (64 channels, into gB2)
  NCU(wgrad(4, net->gC2, net->p2, 64, nullptr, 0, g2));
  NCU(launch_conv(net, net->gC2, 128, nullptr, 0, wbk(net, 4), nullptr, nullptr, net->gB2, 64, false, g2));
  // e2b: pool transpose + skip part of gA1, masked by e2b -> gB1
  combine_kernel<<<grid_for(net, (long long)V1 * 8, 256), 256, 0, net->stream>>>(net->gB2, net->gA1, 192, 128,
                                                                                  net->e2b, net->gB1, 64, g1);
  NCU(cudaGetLastError());
  NCU(wgrad(3, net->gB1, net->e2a, 64, nullptr, 0, g1));
  NCU(launch_conv(net, net->gB1, 64, nullptr, 0, wbk(net, 3), nullptr, net->e2a, net->gC1, 64, false, g1));
  // e2a: gC1 -> gradient of p1 (32 channels, into gB1)
  NCU(wgrad(2, net->gC1, net->p1, 32, nullptr, 0, g1));
  NCU(launch_conv(net, net->gC1, 64, nullptr, 0, wbk(net, 2), nullptr, nullptr, net->gB1, 32, false, g1));
  // e1b: pool transpose + skip part of gA0, masked by e1b -> gB0
  combine_kernel<<<grid_for(net, (long long)V0 * 4, 256), 256, 0, net->stream>>>(net->gB1, net->gA0, 96, 64,
                                                                                  net->e1b, net->gB0, 32, g0);
  NCU(cudaGetLastError());
  NCU(wgrad(1, net->gB0, net->e1a, 32, nullptr, 0, g0));
  NCU(launch_conv(net, net->gB0, 32, nullptr, 0, wbk(net, 1), nullptr, net->e1a, net->gC0, 32, false, g0));
  // e1a (one input channel): its 27 neighbour values as 32 channels (into gA0,
  // free by now), then the weight gradient of one unshifted tap
  im2col_first_kernel<<<grid_for(net, V0, 256), 256, 0, net->stream>>>(v, net->gA0, g0);
  NCU(cudaGetLastError());
  {
    const long long target = (long long)net->num_sms * 8;
    long long z = target;
    const long long zmax = (V0 + 511) / 512;
    if (z > zmax) z = zmax;
    int chunk = (int)(((V0 + z - 1) / z + kWS - 1) / kWS * kWS);
    z = (V0 + chunk - 1) / chunk;
    WgradArgs wa{net->gC0, net->gA0, nullptr, G + T.woff[0], 32, 0, 32, chunk, 1, g0};
    conv_wgrad_kernel<32><<<dim3(1, 1, (unsigned)z), 128, wgrad_smem_bytes<32>(), net->stream>>>(wa);
    NCU(cudaGetLastError());
    NCU(launch_colsum(net, net->gC0, V0, 32, G + T.boff[0]));
  }
  return S3TTV_OK;
}

int pack(s3ttv_net *net) {
  pack_kernel<<<grid_for(net, net->tab.total, 256), 256, 0, net->stream>>>(net->theta, net->tab, net->wf, net->wb,
                                                                           net->hp);
  NCU(cudaGetLastError());
  return S3TTV_OK;
}

int finish(s3ttv_net *net) {
  NCU(cudaStreamSynchronize(net->stream));
  return S3TTV_OK;
}

int gradient_impl(s3ttv_net *net, const float *v, const float *u_ref, const float *s_ref, const float *t_ref, int B,
                  int D, int H, int W, double *loss) {
  int rc = check_shape(net, B, D, H, W);
  if (rc) return rc;
  if (!v || !u_ref || !s_ref || !t_ref) return nfail(net, S3TTV_EINVAL, "null input");
  const Vol g{B, D, H, W};
  const size_t n = (size_t)nvox(g);
  if ((rc = ensure_workspace(net, g))) return rc;
  const float *in[4] = {v, u_ref, s_ref, t_ref}, *dev[4];
  if ((rc = stage_inputs(net, in, 4, n, dev))) return rc;
  if ((rc = run_forward(net, dev[0], g))) return rc;
  if ((rc = run_backward(net, dev[0], dev[1], dev[2], dev[3], g))) return rc;
  if (loss) NCU(cudaMemcpyAsync(loss, net->loss, sizeof(double), cudaMemcpyDeviceToHost, net->stream));
  return S3TTV_OK;
}

}  // namespace

extern "C" {

long long s3ttv_net_param_count(void) { return make_table().total; }

int s3ttv_net_create(s3ttv_net **out, int device, void *stream) {
  if (!out) return S3TTV_EINVAL;
  *out = nullptr;
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess) {
    cudaGetLastError();
    return S3TTV_ECUDA;
  }
  if (device < 0 || device >= ndev) return S3TTV_EINVAL;
  s3ttv_net *net = new (std::nothrow) s3ttv_net();
  if (!net) return S3TTV_ENOMEM;
  net->device = device;
  net->tab = make_table();
  Guard gd(device);
  cudaDeviceGetAttribute(&net->num_sms, cudaDevAttrMultiProcessorCount, device);
  if (net->num_sms <= 0) net->num_sms = 1;
  bool ok = true;
  if (stream) {
    net->stream = (cudaStream_t)stream;
  } else {
    ok = cudaStreamCreateWithFlags(&net->stream, cudaStreamNonBlocking) == cudaSuccess;
    net->own_stream = ok;
  }
  const size_t P = (size_t)net->tab.total;
  ok = ok && cudaMalloc(&net->theta, P * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc(&net->grad, P * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc(&net->m1, P * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc(&net->m2, P * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc(&net->wf, P * sizeof(bf16)) == cudaSuccess;
  ok = ok && cudaMalloc(&net->wb, P * sizeof(bf16)) == cudaSuccess;
  ok = ok && cudaMalloc(&net->hp, (kHeadIn * kHeadOut + kHeadOut) * sizeof(float)) == cudaSuccess;
  ok = ok && cudaMalloc(&net->loss, sizeof(double)) == cudaSuccess;
  if (!ok) {
    cudaGetLastError();
    s3ttv_net_destroy(net);
    return S3TTV_ENOMEM;
  }
  if (cudaFuncSetAttribute(conv_fwd_kernel<128, 64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           conv_smem_bytes<128, 64>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_fwd_kernel<256, 32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           conv_smem_bytes<256, 32>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_wgrad_kernel<128>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           wgrad_smem_bytes<128>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_wgrad_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           wgrad_smem_bytes<64>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_wgrad_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           wgrad_smem_bytes<32>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_wgrad4_kernel<64>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           wgrad4_smem_bytes<64>()) != cudaSuccess ||
      cudaFuncSetAttribute(conv_wgrad4_kernel<32>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                           wgrad4_smem_bytes<32>()) != cudaSuccess) {
    cudaGetLastError();
    s3ttv_net_destroy(net);
    return S3TTV_ECUDA;
  }
  *out = net;
  return S3TTV_OK;
}

void s3ttv_net_destroy(s3ttv_net *net) {
  if (!net) return;
  {
    Guard gd(net->device);
    if (net->stream) cudaStreamSynchronize(net->stream);
    void *bufs[] = {net->theta, net->grad, net->m1, net->m2, net->wf, net->wb, net->hp, net->loss, net->arena,
                    net->stage};
    for (void *b : bufs)
      if (b) cudaFree(b);
    if (net->own_stream) cudaStreamDestroy(net->stream);
  }
  delete net;
}

const char *s3ttv_net_last_error(const s3ttv_net *net) { return net ? net->err : "null network"; }

int s3ttv_net_set_params(s3ttv_net *net, const float *theta) {
  if (!net || !theta) return S3TTV_EINVAL;
  Guard gd(net->device);
  const size_t P = (size_t)net->tab.total;
  NCU(cudaMemcpyAsync(net->theta, theta, P * sizeof(float), cudaMemcpyDefault, net->stream));
  NCU(cudaMemsetAsync(net->m1, 0, P * sizeof(float), net->stream));
  NCU(cudaMemsetAsync(net->m2, 0, P * sizeof(float), net->stream));
  net->adam_t = 0;
  int rc = pack(net);
  if (rc) return rc;
  net->have_params = true;
  return finish(net);
}

int s3ttv_net_get_params(s3ttv_net *net, float *theta) {
  if (!net || !theta) return S3TTV_EINVAL;
  if (!net->have_params) return nfail(net, S3TTV_ESTATE, "parameters not set");
  Guard gd(net->device);
  NCU(cudaMemcpyAsync(theta, net->theta, (size_t)net->tab.total * sizeof(float), cudaMemcpyDefault, net->stream));
  return finish(net);
}

int s3ttv_net_forward(s3ttv_net *net, const float *v, int B, int D, int H, int W, float *u, float *s, float *t) {
  int rc = check_shape(net, B, D, H, W);
  if (rc) return rc;
  if (!v || !u || !s || !t) return nfail(net, S3TTV_EINVAL, "null pointer");
  Guard gd(net->device);
  const Vol g{B, D, H, W};
  const size_t n = (size_t)nvox(g);
  if ((rc = ensure_workspace(net, g))) return rc;
  const float *in[1] = {v}, *dev[1];
  if ((rc = stage_inputs(net, in, 1, n, dev))) return rc;
  if ((rc = run_forward(net, dev[0], g))) return rc;
  float *outs[3] = {u, s, t}, *dout[3];
  const bool host_out = !on_device(u) || !on_device(s) || !on_device(t);
  if (host_out && (rc = ensure_stage(net, 4 * n))) return rc;
  for (int i = 0; i < 3; ++i) dout[i] = on_device(outs[i]) ? outs[i] : net->stage + (size_t)(i + 1) * n;
  head_fwd_kernel<<<grid_for(net, (long long)n, 256), 256, 0, net->stream>>>(net->d1b, dev[0], net->hp, dout[0],
                                                                             dout[1], dout[2], (int)n);
  NCU(cudaGetLastError());
  for (int i = 0; i < 3; ++i)
    if (dout[i] != outs[i])
      NCU(cudaMemcpyAsync(outs[i], dout[i], n * sizeof(float), cudaMemcpyDeviceToHost, net->stream));
  return finish(net);
}

int s3ttv_net_gradient(s3ttv_net *net, const float *v, const float *u_ref, const float *s_ref, const float *t_ref,
                       int B, int D, int H, int W, double *loss, float *grad) {
  if (!net) return S3TTV_EINVAL;
  Guard gd(net->device);
  int rc = gradient_impl(net, v, u_ref, s_ref, t_ref, B, D, H, W, loss);
  if (rc) return rc;
  if (grad)
    NCU(cudaMemcpyAsync(grad, net->grad, (size_t)net->tab.total * sizeof(float), cudaMemcpyDefault, net->stream));
  return finish(net);
}

int s3ttv_net_train_step(s3ttv_net *net, const float *v, const float *u_ref, const float *s_ref, const float *t_ref,
                         int B, int D, int H, int W, float lr, double *loss) {
  if (!net) return S3TTV_EINVAL;
  if (!(lr >= 0.f) || lr > 1.f) return nfail(net, S3TTV_EINVAL, "learning rate %g outside [0, 1]", (double)lr);
  Guard gd(net->device);
  int rc = gradient_impl(net, v, u_ref, s_ref, t_ref, B, D, H, W, loss);
  if (rc) return rc;
  net->adam_t += 1;
  const double b1 = 0.9, b2 = 0.999;
  const float c1 = (float)(1.0 / (1.0 - pow(b1, (double)net->adam_t)));
  const float c2 = (float)(1.0 / (1.0 - pow(b2, (double)net->adam_t)));
  adam_kernel<<<grid_for(net, net->tab.total, 256), 256, 0, net->stream>>>(
      net->theta, net->grad, net->m1, net->m2, net->tab.total, lr, (float)b1, (float)b2, 1e-8f, c1, c2);
  NCU(cudaGetLastError());
  if ((rc = pack(net))) return rc;
  return finish(net);
}

}  // extern "C"
