// Alg. 1 steps 8-11 for the larger blocks the paper itself uses (Sec. IV sets
// the block to 10 x 10 pixels; this file takes k = 6..16, n = k^2 = 36..256
// block rows).  The mathematics is that of block_dual.cu: with
// Y'_l = Y_l + gamma_Y P_l D D_s ubar and G = Y' Y'^T = sum_x lam_x u_x u_x^T,
//
//   Y_l = M Y'_l,   M = I - sum_{lam_x > 1} (1 - lam_x^-1/2) u_x u_x^T,
//
// (eq. prox_nuclear_norm through eq. ProxConjugate: the singular values of Y'_l
// clipped at 1), and Z += P_l^T Y_l.  Only the organisation differs: an n x n
// eigenproblem no longer fits one warp, and a block's Y' (n x 2 N3p floats) no
// longer fits shared memory, so one CTA of kLW warps owns one block at a time
// (a persistent grid strides over the blocks):
//  1. Y' streams through a shared chunk of kCW columns: Y rows plus gamma_Y F
//     (F = D D_s ubar, the cubes Fv, Fh), written back over Y_l for step 5, and
//     accumulated into the Gram by 4 x 4 register tiles of the upper triangle.
//  2. Warm start: C0 = W G from the block's stored normalized eigen-rows W (a
//     NaN marker in W starts cold from C0 = G).
//  3. One-sided (Hestenes) Jacobi on the rows of C, resident in shared memory,
//     in the round-robin ordering: each of the NPOS - 1 steps of a sweep meets
//     NPOS / 2 disjoint row pairs, a group of 8 lanes per pair (4 where that
//     lets one round of the warps cover a step) and 32 / group pairs per warp
//     side by side (a dot product over the group, then the rotation of both
//     rows, held in registers, written back in place); rows never move, only
//     the pairing changes.  Rows are scaled by an exact
//     power of two first; the tolerance, the numerical-zero floor and the
//     rotation formula are those of block_dual.cu.
//  4. Converged rows are lam_x u_x^T: scaled eigen-rows into shared memory, the
//     normalized rows into W for the next pass.
//  5. M = I - Ut^T Ut by 4 x 4 tiles; then Y' streams through the chunk again
//     and every thread forms a 4 x 4 tile of M Y', stored to Y_l and added into
//     Z with float4 atomics.
// The PARTS template parameter sets how many N3p-wide parts a paper-layout row
// has: 2 ([D_v | D_h] differences, S3TTV and STV) or 3 (SSST's first-order
// [D_v u | D_h u | D_s u], F = (Fv, Fh, Fs), Z = (Zv, Zh, Zs)); SSST's k^2 x 3N3
// blocks run here for every k <= kMaxStackedK.
// Above kMaxSmemRows rows (k = 13..16) the two n x n buffers no longer fit
// shared memory: they live in a per-CTA slice of a global scratch (up to
// 2 x 256 x 272 floats, 557 KB per CTA; two CTAs per SM, 72 MB in all at
// k = 13 and 165 MB at k = 16, mostly L2-resident),
// the Gram accumulates its upper-triangle tiles over several passes of the
// chunks (3 tiles a thread per pass) and the Jacobi uses 8-lane groups.
// FP32 throughout (FP32 FMAs on CUDA cores).
#include <math.h>
#include "s3ttv_internal.cuh"

namespace s3ttv {
namespace {

constexpr int kLW = 8;         // warps per CTA (two CTAs per SM where shared memory allows)
constexpr int kLT = kLW * 32;  // threads per CTA
constexpr int kCW = 48;        // columns of Y' per streamed chunk
// The Gram's 4 x 4 tiles read four chunk rows apart (4 (kCW + 4) floats, 16
// banks mod 32) and rotate their column order within 16-column windows.
static_assert(kCW % 16 == 0 && (4 * (kCW + 4)) % 32 == 16, "chunk geometry of the Gram's bank rotation");
// Lanes per row pair in the Jacobi: 8, or 4 where that lets one round of the
// CTA's warps cover every pair of a step (n / 2 pairs) and 8 would need more;
// blocks above kMaxSmemRows rows always 8 (at most 32 floats of a row per lane).
__host__ __device__ constexpr int pair_lanes(int n, int lw) {
  return n > kMaxSmemRows ? 8
                          : (((n + 1) / 2 + lw * 8 - 1) / (lw * 8) < ((n + 1) / 2 + lw * 4 - 1) / (lw * 4) ? 4 : 8);
}

// Two FP32 values in one 64-bit register pair, and the packed FP32x2
// arithmetic of sm_100 and later (each lane rounds as its scalar counterpart).
typedef unsigned long long f32x2;
__device__ __forceinline__ f32x2 pk2(float lo, float hi) {
  f32x2 r;
  asm("mov.b64 %0, {%1, %2};" : "=l"(r) : "f"(lo), "f"(hi));
  return r;
}
__device__ __forceinline__ float2 up2(f32x2 v) {
  float2 r;
  asm("mov.b64 {%0, %1}, %2;" : "=f"(r.x), "=f"(r.y) : "l"(v));
  return r;
}
__device__ __forceinline__ f32x2 fma2(f32x2 a, f32x2 b, f32x2 c) {
  f32x2 r;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(r) : "l"(a), "l"(b), "l"(c));
  return r;
}
__device__ __forceinline__ f32x2 mul2(f32x2 a, f32x2 b) {
  f32x2 r;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(r) : "l"(a), "l"(b));
  return r;
}

struct Layout {
  int n, npos, gs, cs;  // block rows, rows padded to even, row strides of the n x n buffers and the chunk
  int nt4;              // 4-row tiles across npos
  size_t x1, x2, chunk, nrm, pix, last, total;  // float offsets; total floats of shared memory
  size_t rows;          // floats of the n x n buffers in global memory per CTA (0: in shared memory)
};

// n: rows of a block matrix (k^2 in the paper's layout, 2 k^2 stacked).  Above
// kMaxSmemRows rows the two n x n buffers x1, x2 are offsets into the CTA's
// global rows instead of shared memory.
__host__ __device__ inline Layout layout(int n, int pg) {
  Layout L;
  L.n = n;
  L.npos = (L.n + 1) & ~1;
  L.nt4 = (L.npos + 3) / 4;
  const int w = 4 * L.nt4;  // rows and columns rounded to whole tiles
  // a multiple of 4 (float4 rows) and 2 pg mod 32: consecutive rows start
  // 2 pg banks apart, so the pg-lane Jacobi groups of a warp, which read
  // neighbouring rows (2 pg floats each), fill the 32 banks without conflicts
  L.gs = w + (2 * pg - w % 32 + 32) % 32;
  L.cs = kCW + 4;
  L.x1 = 0;
  L.x2 = L.x1 + (size_t)w * L.gs;
  const bool glb = n > kMaxSmemRows;
  L.rows = glb ? L.x2 + (size_t)w * L.gs : 0;
  L.chunk = glb ? 0 : L.x2 + (size_t)w * L.gs;
  L.nrm = L.chunk + (size_t)w * L.cs;
  L.pix = L.nrm + w;
  L.last = L.pix + w;
  L.total = L.last + w;
  return L;
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void sts4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }
__device__ __forceinline__ float c4(const float4 &v, int e) { return e == 0 ? v.x : e == 1 ? v.y : e == 2 ? v.z : v.w; }

// (row, column) of upper-triangle 4 x 4 tile t of an nt4 x nt4 tile grid
__device__ __forceinline__ void upper_tile(int t, int nt4, int &ti, int &tj) {
  ti = 0;
  int left = t, row_len = nt4;
  while (left >= row_len) {
    left -= row_len;
    --row_len;
    ++ti;
  }
  tj = ti + left;
}

// The chunk [c0, c0 + kCW) of Y'_l into shared memory, all 4 nt4 rows (rows
// >= n and columns >= W read as 0).  form: add gamma_Y F and write Y'
// back over Y_l.
// the F cube and band of row r's column c: paper layout, PARTS parts of N3p
// bands per row ([v | h] or SSST's [v | h | s]); stacked, rows 2r, 2r + 1
template <bool ST, int PARTS>
__device__ __forceinline__ const float *f_part(const BlockDualArgs &a, int r, int c, int N3p, int &band) {
  const int part = ST ? (r & 1) : (c >= N3p) + (PARTS == 3 && c >= 2 * N3p);
  band = ST ? c : c - part * N3p;
  return part == 0 ? a.Fv : (part == 1 ? a.Fh : a.Fs);
}
template <bool ST, int PARTS>
__device__ __forceinline__ float *z_part(const BlockDualArgs &a, int r, int c, int N3p, int &band) {
  const int part = ST ? (r & 1) : (c >= N3p) + (PARTS == 3 && c >= 2 * N3p);
  band = ST ? c : c - part * N3p;
  return part == 0 ? a.Zv : (part == 1 ? a.Zh : a.Zs);
}

template <bool ST, int LT, int PARTS>
__device__ void stream_chunk(const Layout &L, float *chunk, float *Yl, const BlockDualArgs &a, const int *pix,
                             int c0, bool form) {
  const Dims &dm = a.dm;
  const int N3p = dm.N3p, W = ST ? N3p : PARTS * N3p;
  constexpr int Q = kCW / 4;
  for (int it = threadIdx.x; it < 4 * L.nt4 * Q; it += LT) {
    const int r = it / Q, q = it - r * Q, c = c0 + 4 * q;
    float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
    if (r < L.n && c < W) {
      float *g = Yl + (size_t)r * W + c;
      y = *reinterpret_cast<const float4 *>(g);
      if (form) {
        int band;
        const float *F = f_part<ST, PARTS>(a, r, c, N3p, band);
        const float4 f = __ldg(reinterpret_cast<const float4 *>(F + (size_t)pix[r] * N3p + band));
        y.x = fmaf(a.gY, f.x, y.x);
        y.y = fmaf(a.gY, f.y, y.y);
        y.z = fmaf(a.gY, f.z, y.z);
        y.w = fmaf(a.gY, f.w, y.w);
        *reinterpret_cast<float4 *>(g) = y;
      }
    }
    sts4(chunk + (size_t)r * L.cs + 4 * q, y);
  }
}

// The same chunk as stream_chunk in two halves, so the next chunk's global
// loads are in flight while the current one is used: fetch_chunk loads this
// thread's PC pieces (Y, and F when forming) into registers, place_chunk forms
// Y' = Y + gamma_Y F, writes it back over Y_l (form) and stores the pieces in
// the chunk (rows >= n and columns >= W as 0).
template <bool ST, int LT, int PARTS, int PC>
__device__ __forceinline__ void fetch_chunk(const Layout &L, const float *Yl, const BlockDualArgs &a, const int *pix,
                                            int c0, bool form, float4 (&y)[PC], float4 (&f)[PC]) {
  const int N3p = a.dm.N3p, W = ST ? N3p : PARTS * N3p;
  constexpr int Q = kCW / 4;
#pragma unroll
  for (int p = 0; p < PC; ++p) {
    const int it = threadIdx.x + p * LT, r = it / Q, q = it - r * Q, c = c0 + 4 * q;
    y[p] = f[p] = make_float4(0.f, 0.f, 0.f, 0.f);
    if (it < 4 * L.nt4 * Q && r < L.n && c < W) {
      y[p] = *reinterpret_cast<const float4 *>(Yl + (size_t)r * W + c);
      if (form) {
        int band;
        const float *F = f_part<ST, PARTS>(a, r, c, N3p, band);
        f[p] = __ldg(reinterpret_cast<const float4 *>(F + (size_t)pix[r] * N3p + band));
      }
    }
  }
}
template <bool ST, int LT, int PARTS, int PC>
__device__ __forceinline__ void place_chunk(const Layout &L, float *chunk, float *Yl, const BlockDualArgs &a, int c0,
                                            bool form, const float4 (&y)[PC], const float4 (&f)[PC]) {
  const int N3p = a.dm.N3p, W = ST ? N3p : PARTS * N3p;
  constexpr int Q = kCW / 4;
#pragma unroll
  for (int p = 0; p < PC; ++p) {
    const int it = threadIdx.x + p * LT, r = it / Q, q = it - r * Q, c = c0 + 4 * q;
    if (it < 4 * L.nt4 * Q) {
      float4 v = y[p];
      if (form) {
        v.x = fmaf(a.gY, f[p].x, v.x);
        v.y = fmaf(a.gY, f[p].y, v.y);
        v.z = fmaf(a.gY, f[p].z, v.z);
        v.w = fmaf(a.gY, f[p].w, v.w);
        if (r < L.n && c < W) *reinterpret_cast<float4 *>(Yl + (size_t)r * W + c) = v;
      }
      sts4(chunk + (size_t)r * L.cs + 4 * q, v);
    }
  }
}

// Column tiles of 8 per unit of the apply's tensor-core loop (a unit: one
// 16-row block of the result over QPU tiles of a chunk of QT tiles, its M
// fragments loaded once per k-step): the largest divisor of QT whose units
// fill the warps' rounds best.
__host__ __device__ constexpr int apply_qpu(int mt, int qt, int lw) {
  int best = 1, best_num = 0, best_den = 1;
  const int cand[4] = {6, 3, 2, 1};
  for (int i = 0; i < 4; ++i) {
    const int q = cand[i];
    if (qt % q) continue;
    const int units = mt * (qt / q), rounds = (units + lw - 1) / lw;
    if ((long long)units * best_den > (long long)best_num * rounds * lw) {  // strictly better filled
      best = q;
      best_num = units;
      best_den = rounds * lw;
    }
  }
  return best;
}

// warps per CTA: stacked blocks of up to 64 rows (k <= 5) and SSST's blocks
// run four-warp CTAs, four per SM; blocks of 101..144 rows, whose two n x n
// matrices fill one SM's shared memory, one sixteen-warp CTA per SM;
// everything else eight-warp CTAs, two per SM
__host__ __device__ constexpr int large_warps_for(int n_rows, bool small) {
  return small ? 4 : (n_rows > 100 && n_rows <= kMaxSmemRows ? 16 : kLW);
}
template <int K, bool ST, int PARTS>
__host__ __device__ constexpr int large_warps() {
  return large_warps_for(ST ? 2 * K * K : K * K, (ST && 2 * K * K <= 64) || (PARTS == 3 && K * K <= 64));
}

template <int K, bool ST, int PARTS>
__global__ void __launch_bounds__(large_warps<K, ST, PARTS>() * 32,
                                  large_warps<K, ST, PARTS>() == 4 ? 4 : (large_warps<K, ST, PARTS>() == 16 ? 1 : 2))
    block_dual_large_kernel(BlockDualArgs a) {
  constexpr int LW = large_warps<K, ST, PARTS>(), LT = LW * 32;
  constexpr int k = K;
  constexpr int NR = ST ? 2 * K * K : K * K;            // rows of a block matrix
  constexpr int NT4 = (((NR + 1) & ~1) + 3) / 4;
  constexpr int GT = (NT4 * (NT4 + 1) / 2 + LT - 1) / LT;  // upper-triangle Gram tiles per thread
  // tiles a thread accumulates per pass over the chunks (more passes above 3)
  constexpr int GTP = GT > 3 ? 3 : GT, NPASS = (GT + GTP - 1) / GTP;
  constexpr int SL = (NR + 31) / 32;                   // row elements a lane holds
  constexpr int PG = pair_lanes(NR, LW);               // lanes per row pair in the Jacobi
  constexpr int PE2 = (NR + 2 * PG - 1) / (2 * PG);    // float2 pieces of a row a Jacobi lane holds
  // skip Jacobi pairs whose rows are unchanged since they last met: pays from
  // about 64 rows (measured: k = 10 3% faster, SSST's 25 rows 8% slower)
  constexpr bool SKIP = NR > 64;
  extern __shared__ __align__(16) float sm[];
  __shared__ float s_red[LW];
  __shared__ unsigned s_sweeps;
  __shared__ int s_queued;  // this block went to the FP64 re-solve
  if (a.sc->done) return;
  const Layout L = layout(NR, PG);
  const int n = L.n, NP = L.npos, GS = L.gs, nt4 = L.nt4;
  float *rb = L.rows ? a.rows + (size_t)blockIdx.x * L.rows : sm;  // where the n x n buffers live
  float *X1 = rb + L.x1, *X2 = rb + L.x2, *chunk = sm + L.chunk, *nrm = sm + L.nrm;
  int *pix = reinterpret_cast<int *>(sm + L.pix);
  int *last = reinterpret_cast<int *>(sm + L.last);  // the last sweep that rotated each Jacobi row
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Dims dm = a.dm;
  const int N3p = dm.N3p, W = ST ? N3p : PARTS * N3p;
  const long long Lb = dm.P;
  if (tid == 0) s_sweeps = 0u;
  const int n_upper = nt4 * (nt4 + 1) / 2;

  for (long long l = blockIdx.x; l < Lb; l += gridDim.x) {
    float *Yl = a.Y + (size_t)l * n * W;
    if (tid < n) {
      const int p = (int)(l / dm.N2), q = (int)(l - (long long)p * dm.N2);
      const int pr = ST ? tid >> 1 : tid;  // window pixel of row tid
      const int ra = pr / k, rc = pr - ra * k;
      int i = p + ra;
      if (i >= dm.N1) i -= dm.N1;
      int j = q + rc;
      if (j >= dm.N2) j -= dm.N2;
      pix[tid] = i * dm.N2 + j;
    }
    __syncthreads();

    // ---- 1. Gram of Y', streamed by column chunks (Y' = Y + gamma_Y F is
    // formed and written back on the first of the NPASS passes; each pass
    // accumulates GTP of a thread's GT upper-triangle tiles) ----
    for (int ps = 0; ps < NPASS; ++ps) {
    float acc[GTP][16];
#pragma unroll
    for (int u = 0; u < GTP; ++u)
#pragma unroll
      for (int e = 0; e < 16; ++e) acc[u][e] = 0.f;
    // Blocks of fewer than 64 rows (their Gram is bound by streaming the
    // chunks, measured) fetch the next chunk into registers while this one's
    // products run; larger ones would spill (two CTAs per SM) and stream as is.
    constexpr int PC = (4 * NT4 * (kCW / 4) + LT - 1) / LT;
    constexpr bool PREF = PC <= 6 && NR < 64;
    constexpr int PCR = PREF ? PC : 1;
    float4 ry[PCR], rf[PCR];
    if constexpr (PREF) fetch_chunk<ST, LT, PARTS, PCR>(L, Yl, a, pix, 0, ps == 0, ry, rf);
    for (int c0 = 0; c0 < W; c0 += kCW) {
      if constexpr (PREF) {
        place_chunk<ST, LT, PARTS, PCR>(L, chunk, Yl, a, c0, ps == 0, ry, rf);
      } else {
        stream_chunk<ST, LT, PARTS>(L, chunk, Yl, a, pix, c0, ps == 0);
      }
      __syncthreads();
      if constexpr (PREF)
        if (c0 + kCW < W) fetch_chunk<ST, LT, PARTS, PCR>(L, Yl, a, pix, c0 + kCW, ps == 0, ry, rf);
#pragma unroll
      for (int u = 0; u < GTP; ++u) {
        const int t = tid + (ps * GTP + u) * LT;
        if (t < n_upper) {
          int ti, tj;
          upper_tile(t, nt4, ti, tj);
          const float *pa = chunk + (size_t)(4 * ti) * L.cs, *pb = chunk + (size_t)(4 * tj) * L.cs;
          // the 8 lanes of a quarter-warp hold consecutive tj, whose B rows
          // start 0 or 16 banks apart: rotating the column order by
          // 4 ((tj / 2) mod 4) within each 16-column window puts their
          // float4 loads on 8 distinct 4-bank groups (the sums only reorder)
          const int rot = 4 * ((tj >> 1) & 3);
#pragma unroll 2
          for (int c = 0; c < kCW; c += 4) {
            const int cc = (c & ~15) | ((c + rot) & 15);
            float4 va[4], vb[4];
#pragma unroll
            for (int x = 0; x < 4; ++x) {
              va[x] = lds4(pa + (size_t)x * L.cs + cc);
              vb[x] = lds4(pb + (size_t)x * L.cs + cc);
            }
#pragma unroll
            for (int x = 0; x < 4; ++x)
#pragma unroll
              for (int y = 0; y < 4; ++y) {
                float s = acc[u][4 * x + y];
                s = fmaf(va[x].x, vb[y].x, s);
                s = fmaf(va[x].y, vb[y].y, s);
                s = fmaf(va[x].z, vb[y].z, s);
                s = fmaf(va[x].w, vb[y].w, s);
                acc[u][4 * x + y] = s;
              }
          }
        }
      }
      __syncthreads();
    }
#pragma unroll
    for (int u = 0; u < GTP; ++u) {
      const int t = tid + (ps * GTP + u) * LT;
      if (t < n_upper) {
        int ti, tj;
        upper_tile(t, nt4, ti, tj);
#pragma unroll
        for (int x = 0; x < 4; ++x)
#pragma unroll
          for (int y = 0; y < 4; ++y) {
            const int r = 4 * ti + x, c = 4 * tj + y;
            X1[(size_t)r * GS + c] = acc[u][4 * x + y];
            X1[(size_t)c * GS + r] = acc[u][4 * x + y];
          }
      }
    }
    }  // passes
    __syncthreads();

    // ---- 2. C0 = W G (warm) or G (cold), rows of C into X2 ----
    const float *Wl = a.W ? a.W + (size_t)l * a.w_stride : nullptr;
    const bool warm = a.warm && Wl && !(Wl[0] != Wl[0]);  // NaN marks "start cold"
    bool c0_done = false;
    if constexpr (NR >= 64) {
      if (warm) {  // block-uniform
        // C0 = W G on the tensor cores (three TF32 products per FP32 product):
        // unit u = rows 16 m .. 16 m + 15 of C0 over Q0 column tiles of 8, W's
        // fragments (from global memory) loaded once per k-step for all of them
        constexpr int NPC = (NR + 1) & ~1, MT0 = (NPC + 15) / 16, QT0 = (NR + 7) / 8, KS0 = (NR + 7) / 8;
        constexpr int G0 = (QT0 + 6) / 7, Q0 = (QT0 + G0 - 1) / G0, UNITS0 = MT0 * G0;
        const int g = lane >> 2, t = lane & 3;
        for (int e = tid; e < NP * (GS - 8 * QT0); e += LT) {  // columns beyond the tiles
          const int r = e / (GS - 8 * QT0);
          X2[(size_t)r * GS + 8 * QT0 + (e - r * (GS - 8 * QT0))] = 0.f;
        }
        for (int u = warp; u < UNITS0; u += LW) {
          const int m = u / G0, q0 = (u - m * G0) * Q0;
          float d[Q0][4];
#pragma unroll
          for (int qq = 0; qq < Q0; ++qq) d[qq][0] = d[qq][1] = d[qq][2] = d[qq][3] = 0.f;
#pragma unroll 2
          for (int ks = 0; ks < KS0; ++ks) {
            unsigned ah[4], al[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int i = 16 * m + g + 8 * (e & 1), k = 8 * ks + t + 4 * (e >> 1);
              split_tf32(i < NP && k < n ? __ldg(Wl + (size_t)i * n + k) : 0.f, ah[e], al[e]);
            }
            unsigned bh[Q0][2], bl[Q0][2];
#pragma unroll
            for (int qq = 0; qq < Q0; ++qq)
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int k = 8 * ks + t + 4 * h, j = 8 * (q0 + qq) + g;
                split_tf32(k < n && j < n && q0 + qq < QT0 ? X1[(size_t)k * GS + j] : 0.f, bh[qq][h], bl[qq][h]);
              }
            three_parts([&](auto P) {
#pragma unroll
              for (int qq = 0; qq < Q0; ++qq)
                mma_3xtf32_part<decltype(P)::value>(d[qq], ah, al, bh[qq][0], bh[qq][1], bl[qq][0], bl[qq][1]);
            });
          }
#pragma unroll
          for (int qq = 0; qq < Q0; ++qq) {
            if (q0 + qq >= QT0) break;
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int r = 16 * m + g + 8 * h;
              if (r < NP)
                *reinterpret_cast<float2 *>(X2 + (size_t)r * GS + 8 * (q0 + qq) + 2 * t) =
                    make_float2(d[qq][2 * h], d[qq][2 * h + 1]);
            }
          }
        }
        c0_done = true;
      }
    }
    // two rows per warp at a time (r0 and r0 + LW), so each G row loaded from
    // shared memory serves both; per row the sums are those of one row at a time
    for (int r0 = warp; r0 < NP && !c0_done; r0 += 2 * LW) {
      const int r1 = r0 + LW;
      const bool two = r1 < NP;
      float acc0[SL], acc1[SL];
      if (warm) {
        float w0[SL], w1[SL];  // lane j holds W[r][j + 32 i]
#pragma unroll
        for (int i = 0; i < SL; ++i) {
          const int c = lane + 32 * i;
          w0[i] = c < n ? __ldg(Wl + (size_t)r0 * n + c) : 0.f;
          w1[i] = two && c < n ? __ldg(Wl + (size_t)r1 * n + c) : 0.f;
          acc0[i] = 0.f;
          acc1[i] = 0.f;
        }
#pragma unroll
        for (int kb = 0; kb < SL; ++kb) {
          for (int j = 0; j < 32 && kb * 32 + j < n; ++j) {
            const float wa = __shfl_sync(kFull, w0[kb], j), wb = __shfl_sync(kFull, w1[kb], j);
            const float *g = X1 + (size_t)(kb * 32 + j) * GS;
#pragma unroll
            for (int i = 0; i < SL; ++i) {
              const int c = lane + 32 * i;
              if (c < n) {
                const float gv = g[c];
                acc0[i] = fmaf(wa, gv, acc0[i]);
                acc1[i] = fmaf(wb, gv, acc1[i]);
              }
            }
          }
        }
      } else {
#pragma unroll
        for (int i = 0; i < SL; ++i) {
          const int c = lane + 32 * i;
          acc0[i] = r0 < n && c < n ? X1[(size_t)r0 * GS + c] : 0.f;
          acc1[i] = r1 < n && c < n ? X1[(size_t)r1 * GS + c] : 0.f;
        }
      }
#pragma unroll
      for (int i = 0; i < SL; ++i) {
        const int c = lane + 32 * i;
        if (c < GS) {
          X2[(size_t)r0 * GS + c] = c < n ? acc0[i] : 0.f;
          if (two) X2[(size_t)r1 * GS + c] = c < n ? acc1[i] : 0.f;
        }
      }
    }
    __syncthreads();

    // ---- 3. one-sided Jacobi on the rows of C ----
    if (SKIP)
      for (int r = tid; r < NP; r += LT) last[r] = -2;  // published by the barrier in norms()
    // squared row norms (one warp per row)
    auto norms = [&]() {
      for (int r = warp; r < NP; r += LW) {
        float s = 0.f;
        for (int c = lane; c < n; c += 32) s = fmaf(X2[(size_t)r * GS + c], X2[(size_t)r * GS + c], s);
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
        if (lane == 0) nrm[r] = s;
      }
      __syncthreads();
    };
    norms();
    // every warp sums the same norms in the same order: a block-uniform value
    float fro = 0.f;
    for (int r = lane; r < NP; r += 32) fro += nrm[r];
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(kFull, fro, o);
    // exact power-of-two scaling to a Frobenius norm near 1; eigenvalues are
    // unscaled at the end by inv_s
    float inv_s = 1.f;
    if (fro > 0.f && fro < 1e30f) {
      const int ex = ((__float_as_int(fro) >> 23) & 255) - 127;
      const int h = ex >> 1;
      const float sc = __int_as_float((127 - h) << 23), sc2 = sc * sc;
      inv_s = __int_as_float((127 + h) << 23);
      __syncthreads();  // every warp has read nrm for fro
      for (int e = tid; e < NP * GS; e += LT) X2[e] *= sc;
      for (int r = tid; r < NP; r += LT) nrm[r] *= sc2;
      fro *= sc2;
      __syncthreads();
    }
    const float floor2 = 1e-12f * fro;
    const float tol2 = a.tol * a.tol, pol2 = a.polish * a.polish;
    bool converged = false;
    int sweeps = 0;
    for (int sw = 0; sw < a.max_sweeps; ++sw) {
      if (sw) norms();
      int rotated = 0;
      for (int step = 0; step < NP - 1; ++step) {
        // PG lanes per pair, 32 / PG pairs per warp side by side
        for (int base = 0; base < NP / 2; base += LW * (32 / PG)) {
          if (base + warp * (32 / PG) >= NP / 2) continue;  // the whole warp has no pair this round
          const int i = base + warp * (32 / PG) + (lane / PG), gl = lane % PG;
          const bool act = i < NP / 2;
          // round robin: position 0 fixed, positions 1..NP-1 turn by one each step
          const int pa = act ? i : 0, pb = NP - 1 - pa;
          int xa = pa - 1 + step, xb = pb - 1 + step;  // both < 2 (NP - 1)
          xa -= xa >= NP - 1 ? NP - 1 : 0;
          xb -= xb >= NP - 1 ? NP - 1 : 0;
          const int ra = pa == 0 ? 0 : 1 + xa, rb = 1 + xb;
          float *A = X2 + (size_t)ra * GS, *B = X2 + (size_t)rb * GS;
          // a pair whose rows no rotation has touched since the pair last met
          // (in the previous sweep, with the same rows, and did not rotate
          // then) would compute the same product: it is skipped
          const bool chk = act && (!SKIP || sw == 0 || last[ra] >= sw - 1 || last[rb] >= sw - 1);
          if (SKIP && !__any_sync(kFull, chk)) continue;  // warp-uniform
          // lane gl holds the float2 pieces at columns 2 gl + 2 PG e; columns
          // n..GS-1 of every row are zero, so a piece starting below n is whole
          f32x2 va[PE2], vb[PE2];
          f32x2 dd = 0ull;
#pragma unroll
          for (int e = 0; e < PE2; ++e) {
            const int c = 2 * gl + 2 * PG * e;
            const bool in = chk && c < n;
            va[e] = in ? *reinterpret_cast<const f32x2 *>(A + c) : 0ull;
            vb[e] = in ? *reinterpret_cast<const f32x2 *>(B + c) : 0ull;
            dd = fma2(va[e], vb[e], dd);
          }
          const float2 d2 = up2(dd);
          float d = d2.x + d2.y;
#pragma unroll
          for (int o = PG / 2; o > 0; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
          const float nA = chk ? nrm[ra] : 0.f, nB = chk ? nrm[rb] : 0.f;
          if (chk && fminf(nA, nB) > floor2 && d * d > pol2 * nA * nB) {
            const float x = nB - nA, y = 2.f * d;
            const float rr = rsqrtf(fmaf(x, x, y * y));
            const float hc = fmaf(0.5f * fabsf(x), rr, 0.5f);
            const float rc = rsqrtf(hc);
            const float cs = hc * rc, sn = copysignf(0.5f, x) * y * rr * rc;
            const float dn = sn * rc * d;  // t apq
            const f32x2 cs2 = pk2(cs, cs), sn2 = pk2(sn, sn), ns2 = pk2(-sn, -sn);
#pragma unroll
            for (int e = 0; e < PE2; ++e) {
              const int c = 2 * gl + 2 * PG * e;
              if (c < n) {
                *reinterpret_cast<f32x2 *>(A + c) = fma2(cs2, va[e], mul2(ns2, vb[e]));
                *reinterpret_cast<f32x2 *>(B + c) = fma2(sn2, va[e], mul2(cs2, vb[e]));
              }
            }
            if (gl == 0) {
              nrm[ra] = nA - dn;
              nrm[rb] = nB + dn;
              if (SKIP) {
                last[ra] = sw;
                last[rb] = sw;
              }
            }
            if (d * d > tol2 * nA * nB) rotated = 1;
          }
        }
        __syncthreads();
      }
      ++sweeps;
      if (!__syncthreads_or(rotated)) {
        converged = true;
        break;
      }
    }
    if (tid == 0) {
      int queued = 0;
      if (!converged) {
        // to the FP64 re-solve if the queue has room; else applied as it stands
        const unsigned slot = a.fb_list ? atomicAdd(&a.sc->fb_count, 1u) : 0xffffffffu;
        if (slot < (unsigned)a.fb_cap) {
          a.fb_list[slot] = (int)l;
          queued = 1;
        } else {
          atomicAdd(&a.sc->jacobi_fail, 1u);
        }
      }
      s_queued = queued;
      s_sweeps += (unsigned)sweeps;
    }
    norms();  // ends with a barrier: s_queued is visible
    if (s_queued) continue;  // CTA-uniform: Y_l keeps Y' (written back in the Gram pass), no Z

    // ---- 4. eigen-rows: Ut (X1), and the unit eigenvectors in place in X2 ----
    for (int r = warp; r < NP; r += LW) {
      const float nr = nrm[r];
      const float lam = sqrtf(nr) * inv_s;
      const float wt = lam > 1.f ? sqrtf(1.f - rsqrtf(lam)) * rsqrtf(nr) : 0.f;
      const float inr = nr > floor2 ? rsqrtf(nr) : 0.f;
      for (int c = lane; c < GS; c += 32) {
        const float v = c < n ? X2[(size_t)r * GS + c] : 0.f;
        X1[(size_t)r * GS + c] = v * wt;
        X2[(size_t)r * GS + c] = v * inr;
      }
    }
    __syncthreads();

    // ---- 4b. the warm rows W: the eigenvectors completed to an orthonormal basis ----
    // Rows below the numerical-zero floor carry no reliable direction; each
    // needs a unit vector that completes the converged rows to an orthonormal
    // basis.  A warm pass takes the block's stored W rows at those positions
    // and finishes with Jacobi sweeps over the same round-robin ordering with
    // the converged rows frozen: a pair of a frozen row and a candidate
    // projects the candidate off the frozen row, two candidates rotate as in
    // step 3, two frozen rows are skipped (the eigen-rows, and so M, are those
    // of step 3).  The rank deficiency is often structural and the same every
    // pass (the stacked blocks of k x k windows have the (k - 1)^2 discrete
    // curl relations of their vertical and horizontal differences), so the
    // stored rows already complete the basis.  A cold pass, a candidate left
    // with no more than 1 / (2 n) of its squared norm, or sweeps that do not
    // converge fall back to Gram-Schmidt: each missing row is the first unit
    // vector e_j whose remainder against every unit row so far (classical
    // Gram-Schmidt, twice) keeps more than 1 / (2 n) of its squared norm (the
    // largest remainder is at least 1 / n while the rows span less than R^n).
    // The block is marked cold only if that fails too.
    if (a.W) {
      float *xv = chunk, *coef = chunk + GS;  // the chunk is free until the apply
      int below = 0;
      for (int r = tid; r < n; r += LT) below |= nrm[r] <= floor2 ? 1 : 0;
      bool cold = false;
      if (__syncthreads_or(below)) {  // block-uniform
        for (int r = tid; r < NP; r += LT) last[r] = r >= n || nrm[r] > floor2 ? 1 : 0;
        __syncthreads();
        bool ok = false;
        if (warm) {
          for (int r = warp; r < NP; r += LW)
            if (!last[r])
              for (int c = lane; c < GS; c += 32) X2[(size_t)r * GS + c] = c < n ? __ldg(Wl + (size_t)r * n + c) : 0.f;
          __syncthreads();
          norms();  // frozen rows 1 (0 for a padding row), candidates their own
          bool done = false;
          for (int sw = 0; sw < a.max_sweeps && !done; ++sw) {
            if (sw) norms();
            int rotated = 0;
            for (int step = 0; step < NP - 1; ++step) {
              for (int base = 0; base < NP / 2; base += LW * (32 / PG)) {
                if (base + warp * (32 / PG) >= NP / 2) continue;
                const int i = base + warp * (32 / PG) + (lane / PG), gl = lane % PG;
                const bool act = i < NP / 2;
                const int pa = act ? i : 0, pb = NP - 1 - pa;
                int xa = pa - 1 + step, xb = pb - 1 + step;
                xa -= xa >= NP - 1 ? NP - 1 : 0;
                xb -= xb >= NP - 1 ? NP - 1 : 0;
                const int ra = pa == 0 ? 0 : 1 + xa, rb = 1 + xb;
                const int fa = act ? last[ra] : 1, fb = act ? last[rb] : 1;
                const bool chk = !(fa && fb);
                if (!__any_sync(kFull, chk)) continue;  // warp-uniform
                float *A = X2 + (size_t)ra * GS, *B = X2 + (size_t)rb * GS;
                f32x2 va[PE2], vb[PE2];
                f32x2 dd = 0ull;
#pragma unroll
                for (int e = 0; e < PE2; ++e) {
                  const int c = 2 * gl + 2 * PG * e;
                  const bool in = chk && c < n;
                  va[e] = in ? *reinterpret_cast<const f32x2 *>(A + c) : 0ull;
                  vb[e] = in ? *reinterpret_cast<const f32x2 *>(B + c) : 0ull;
                  dd = fma2(va[e], vb[e], dd);
                }
                const float2 d2 = up2(dd);
                float d = d2.x + d2.y;
#pragma unroll
                for (int o = PG / 2; o > 0; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
                const float nA = chk ? nrm[ra] : 0.f, nB = chk ? nrm[rb] : 0.f;
                if (chk && fminf(nA, nB) > 1e-12f && d * d > pol2 * nA * nB) {
                  if (fa || fb) {  // the candidate minus its component along the frozen row
                    float *Cr = fa ? B : A;
                    const float nf = fa ? nA : nB, m = -d / nf;
                    const f32x2 m2 = pk2(m, m);
#pragma unroll
                    for (int e = 0; e < PE2; ++e) {
                      const int c = 2 * gl + 2 * PG * e;
                      if (c < n) *reinterpret_cast<f32x2 *>(Cr + c) = fa ? fma2(m2, va[e], vb[e]) : fma2(m2, vb[e], va[e]);
                    }
                    if (gl == 0) nrm[fa ? rb : ra] = (fa ? nB : nA) + m * d;
                  } else {
                    const float x = nB - nA, y = 2.f * d;
                    const float rr = rsqrtf(fmaf(x, x, y * y));
                    const float hc = fmaf(0.5f * fabsf(x), rr, 0.5f);
                    const float rc = rsqrtf(hc);
                    const float cs = hc * rc, sn = copysignf(0.5f, x) * y * rr * rc;
                    const float dn = sn * rc * d;
                    const f32x2 cs2 = pk2(cs, cs), sn2 = pk2(sn, sn), ns2 = pk2(-sn, -sn);
#pragma unroll
                    for (int e = 0; e < PE2; ++e) {
                      const int c = 2 * gl + 2 * PG * e;
                      if (c < n) {
                        *reinterpret_cast<f32x2 *>(A + c) = fma2(cs2, va[e], mul2(ns2, vb[e]));
                        *reinterpret_cast<f32x2 *>(B + c) = fma2(sn2, va[e], mul2(cs2, vb[e]));
                      }
                    }
                    if (gl == 0) {
                      nrm[ra] = nA - dn;
                      nrm[rb] = nB + dn;
                    }
                  }
                  if (d * d > tol2 * nA * nB) rotated = 1;
                }
              }
              __syncthreads();
            }
            done = !__syncthreads_or(rotated);
          }
          norms();
          ok = done;  // block-uniform: every thread reads the same norms after the barrier
          for (int r = 0; r < n; ++r)
            if (!last[r] && nrm[r] * (float)(2 * n) <= 1.f) ok = false;
          if (ok) {
            for (int r = warp; r < n; r += LW) {
              if (last[r]) continue;
              const float sc = rsqrtf(nrm[r]);
              for (int c = lane; c < n; c += 32) X2[(size_t)r * GS + c] *= sc;
            }
          }
        }
        if (!ok) {  // Gram-Schmidt from unit vectors: missing rows zero, unit rows marked by nrm
          for (int r = warp; r < NP; r += LW) {
            if (!last[r])
              for (int c = lane; c < GS; c += 32) X2[(size_t)r * GS + c] = 0.f;
            if (lane == 0) nrm[r] = last[r] && r < n ? 1.f : 0.f;
          }
          __syncthreads();
          int next_e = 0;
          for (int r = 0; r < n && !cold; ++r) {
            if (nrm[r] > floor2) continue;  // block-uniform: shared memory read after a barrier
            bool placed = false;
            while (!placed && next_e < n) {
              const int j = next_e++;
              for (int c = tid; c < n; c += LT) xv[c] = c == j ? 1.f : 0.f;
              __syncthreads();
              for (int pass = 0; pass < 2; ++pass) {
                for (int s2 = warp; s2 < n; s2 += LW) {
                  float d = 0.f;
                  if (nrm[s2] > floor2)
                    for (int c = lane; c < n; c += 32) d = fmaf(X2[(size_t)s2 * GS + c], xv[c], d);
#pragma unroll
                  for (int o = 16; o > 0; o >>= 1) d += __shfl_xor_sync(kFull, d, o);
                  if (lane == 0) coef[s2] = d;
                }
                __syncthreads();
                for (int c = tid; c < n; c += LT) {
                  float x = xv[c];
                  for (int s2 = 0; s2 < n; ++s2) x = fmaf(-coef[s2], X2[(size_t)s2 * GS + c], x);
                  xv[c] = x;
                }
                __syncthreads();
              }
              float q = 0.f;
              for (int c = tid; c < n; c += LT) q = fmaf(xv[c], xv[c], q);
#pragma unroll
              for (int o = 16; o > 0; o >>= 1) q += __shfl_xor_sync(kFull, q, o);
              if (lane == 0) s_red[warp] = q;
              __syncthreads();
              q = 0.f;
              for (int w = 0; w < LW; ++w) q += s_red[w];
              if (q * (float)(2 * n) > 1.f) {
                const float iq = rsqrtf(q);
                for (int c = tid; c < GS; c += LT) X2[(size_t)r * GS + c] = c < n ? xv[c] * iq : 0.f;
                if (tid == 0) nrm[r] = 1.f;  // a unit row from now on
                placed = true;
              }
              __syncthreads();
            }
            if (!placed) cold = true;
          }
        }
        __syncthreads();
      }
      if (!cold) {
        for (int r = warp; r < NP; r += LW) {
          float *ww = a.W + (size_t)l * a.w_stride + (size_t)r * n;
          for (int c = lane; c < n; c += 32) ww[c] = X2[(size_t)r * GS + c];
        }
      }
      __syncthreads();  // every W row written (and X2 read) before the marker and before M takes X2's place
      if (cold && tid == 0) a.W[(size_t)l * a.w_stride] = __int_as_float(0x7fc00000);
    }

    // ---- 5a. M = I - Ut^T Ut into X2: upper-triangle 4 x 4 tiles, each
    // written with its transpose (M is symmetric) ----
    for (int t = tid; t < n_upper; t += LT) {
      int ti, tj;
      upper_tile(t, nt4, ti, tj);
      float m[16];
#pragma unroll
      for (int e = 0; e < 16; ++e) m[e] = 0.f;
      for (int x = 0; x < NP; ++x) {
        const float4 ua = lds4(X1 + (size_t)x * GS + 4 * ti), ub = lds4(X1 + (size_t)x * GS + 4 * tj);
#pragma unroll
        for (int p = 0; p < 4; ++p)
#pragma unroll
          for (int q = 0; q < 4; ++q) m[4 * p + q] = fmaf(c4(ua, p), c4(ub, q), m[4 * p + q]);
      }
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const int r = 4 * ti + p;
        sts4(X2 + (size_t)r * GS + 4 * tj,
             make_float4((r == 4 * tj ? 1.f : 0.f) - m[4 * p], (r == 4 * tj + 1 ? 1.f : 0.f) - m[4 * p + 1],
                         (r == 4 * tj + 2 ? 1.f : 0.f) - m[4 * p + 2], (r == 4 * tj + 3 ? 1.f : 0.f) - m[4 * p + 3]));
      }
      if (ti != tj) {
#pragma unroll
        for (int q = 0; q < 4; ++q)  // row 4 tj + q of the transpose: off the diagonal, no identity
          sts4(X2 + (size_t)(4 * tj + q) * GS + 4 * ti, make_float4(-m[q], -m[4 + q], -m[8 + q], -m[12 + q]));
      }
    }
    __syncthreads();

    // ---- 5b. Y_l = M Y' by chunks; Z += P_l^T Y_l.  Blocks of at least 64
    // rows on the tensor cores (three TF32 products per FP32 product); smaller
    // ones, whose apply is bound by streaming the chunks rather than by the
    // products (measured), by 4 x 4 FP32 register tiles ----
    if constexpr (NR < 64) {
      // the next chunk of Y' is fetched into registers while this one is applied
      constexpr int PC = (4 * NT4 * (kCW / 4) + LT - 1) / LT;
      constexpr bool PREF = PC <= 6;
      constexpr int PCR = PREF ? PC : 1;
      float4 ry[PCR], rf[PCR];
      if constexpr (PREF) fetch_chunk<ST, LT, PARTS, PCR>(L, Yl, a, pix, 0, false, ry, rf);
      for (int c0 = 0; c0 < W; c0 += kCW) {
        if constexpr (PREF) {
          place_chunk<ST, LT, PARTS, PCR>(L, chunk, Yl, a, c0, false, ry, rf);
        } else {
          stream_chunk<ST, LT, PARTS>(L, chunk, Yl, a, pix, c0, false);
        }
        __syncthreads();
        if constexpr (PREF)
          if (c0 + kCW < W) fetch_chunk<ST, LT, PARTS, PCR>(L, Yl, a, pix, c0 + kCW, false, ry, rf);
        constexpr int Q = kCW / 4;
        for (int t = tid; t < nt4 * Q; t += LT) {
          const int ti = t / Q, q = t - ti * Q;
          float4 y[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) y[p] = make_float4(0.f, 0.f, 0.f, 0.f);
          for (int s = 0; s < n; ++s) {
            const float4 m = lds4(X2 + (size_t)s * GS + 4 * ti);  // M[s][r] = M[r][s]
            const float4 v = lds4(chunk + (size_t)s * L.cs + 4 * q);
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const float mp = c4(m, p);
              y[p].x = fmaf(mp, v.x, y[p].x);
              y[p].y = fmaf(mp, v.y, y[p].y);
              y[p].z = fmaf(mp, v.z, y[p].z);
              y[p].w = fmaf(mp, v.w, y[p].w);
            }
          }
          const int c = c0 + 4 * q;
          if (c < W) {
#pragma unroll
            for (int p = 0; p < 4; ++p) {
              const int r = 4 * ti + p;
              if (r < n) {
                int band;
                float *Zb = z_part<ST, PARTS>(a, r, c, N3p, band);
                __stcs(reinterpret_cast<float4 *>(Yl + (size_t)r * W + c), y[p]);
                atomicAdd(reinterpret_cast<float4 *>(Zb + (size_t)pix[r] * N3p + band), y[p]);
              }
            }
          }
        }
        __syncthreads();
      }
    } else {
    // M's low TF32 parts into X1 (Ut is no longer read); X2 keeps M, whose raw
    // bits are its high parts.  A = M read transposed (M is symmetric).
    for (int e = tid; e < n * GS; e += LT) {
      const float m = X2[e];
      X1[e] = m - __uint_as_float(__float_as_uint(m) & 0xffffe000u);
    }
    __syncthreads();
    {
      constexpr int MT = (NR + 15) / 16, KS = (NR + 7) / 8, QT = kCW / 8;
      constexpr int QPU = apply_qpu(MT, QT, LW), UPR = QT / QPU, UNITS = MT * UPR;
      constexpr int ROUNDS = (UNITS + LW - 1) / LW;
      const int g = lane >> 2, t = lane & 3;
      for (int c0 = 0; c0 < W; c0 += kCW) {
        stream_chunk<ST, LT, PARTS>(L, chunk, Yl, a, pix, c0, false);
        __syncthreads();
        // unit u: rows 16 m .. 16 m + 15 of the chunk's result, QPU column tiles of 8
        float d[ROUNDS][QPU][4];
#pragma unroll
        for (int rd = 0; rd < ROUNDS; ++rd) {
#pragma unroll
          for (int qq = 0; qq < QPU; ++qq) d[rd][qq][0] = d[rd][qq][1] = d[rd][qq][2] = d[rd][qq][3] = 0.f;
          const int u = warp + rd * LW;
          if (u >= UNITS) continue;  // warp-uniform
          const int m = u / UPR, q0 = (u - m * UPR) * QPU;
#pragma unroll 2
          for (int ks = 0; ks < KS; ++ks) {
            unsigned ah[4], al[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int i = 16 * m + g + 8 * (e & 1), k = 8 * ks + t + 4 * (e >> 1);
              const bool in = i < n && k < n;
              ah[e] = in ? __float_as_uint(X2[(size_t)k * GS + i]) : 0u;
              al[e] = in ? __float_as_uint(X1[(size_t)k * GS + i]) : 0u;
            }
            unsigned bh[QPU][2], bl[QPU][2];
#pragma unroll
            for (int qq = 0; qq < QPU; ++qq)
#pragma unroll
              for (int h = 0; h < 2; ++h) {
                const int k = 8 * ks + t + 4 * h;
                split_tf32(k < n ? chunk[(size_t)k * L.cs + 8 * (q0 + qq) + g] : 0.f, bh[qq][h], bl[qq][h]);
              }
            three_parts([&](auto P) {
#pragma unroll
              for (int qq = 0; qq < QPU; ++qq)
                mma_3xtf32_part<decltype(P)::value>(d[rd][qq], ah, al, bh[qq][0], bh[qq][1], bl[qq][0], bl[qq][1]);
            });
          }
        }
        __syncthreads();  // every warp has read the chunk: the results take its place
#pragma unroll
        for (int rd = 0; rd < ROUNDS; ++rd) {
          const int u = warp + rd * LW;
          if (u >= UNITS) continue;
          const int m = u / UPR, q0 = (u - m * UPR) * QPU;
#pragma unroll
          for (int qq = 0; qq < QPU; ++qq)
#pragma unroll
            for (int h = 0; h < 2; ++h) {
              const int r = 16 * m + g + 8 * h;
              if (r < n)
                *reinterpret_cast<float2 *>(chunk + (size_t)r * L.cs + 8 * (q0 + qq) + 2 * t) =
                    make_float2(d[rd][qq][2 * h], d[rd][qq][2 * h + 1]);
            }
        }
        __syncthreads();
        constexpr int Q = kCW / 4;
        for (int it = tid; it < n * Q; it += LT) {
          const int r = it / Q, j = it - r * Q, c = c0 + 4 * j;
          if (c < W) {
            const float4 y = lds4(chunk + (size_t)r * L.cs + 4 * j);
            int band;
            float *Zb = z_part<ST, PARTS>(a, r, c, N3p, band);
            __stcs(reinterpret_cast<float4 *>(Yl + (size_t)r * W + c), y);
            atomicAdd(reinterpret_cast<float4 *>(Zb + (size_t)pix[r] * N3p + band), y);
          }
        }
        __syncthreads();
      }
    }
    }  // tensor-core apply
  }
  if (tid == 0 && s_sweeps) atomicAdd(&a.sc->jacobi_sweeps, (unsigned long long)s_sweeps);
}

}  // namespace

size_t block_dual_large_smem_bytes(int k, bool stacked, int parts) {
  const int n = stacked ? 2 * k * k : k * k;
  return sizeof(float) * layout(n, pair_lanes(n, block_dual_large_threads(k, stacked, parts) / 32)).total;
}

size_t block_dual_large_rows_floats(int k, bool stacked, int parts) {
  const int n = stacked ? 2 * k * k : k * k;
  return layout(n, pair_lanes(n, block_dual_large_threads(k, stacked, parts) / 32)).rows;
}

long long block_dual_large_w_stride(int k, bool stacked) {
  const Layout L = layout(stacked ? 2 * k * k : k * k, 8);  // npos and n only
  return ((long long)L.npos * L.n + 3) / 4 * 4;
}

long long block_dual_large_w_stride(int k) { return block_dual_large_w_stride(k, false); }

int block_dual_large_threads(int k, bool stacked, int parts) {
  const int n = stacked ? 2 * k * k : k * k;
  return 32 * large_warps_for(n, (stacked && n <= 64) || (parts == 3 && k * k <= 64));
}

namespace {
typedef void (*LargeKernel)(BlockDualArgs);
LargeKernel large_kernel(int k, bool stacked, int parts) {
  static const LargeKernel paper[] = {block_dual_large_kernel<6, false, 2>,  block_dual_large_kernel<7, false, 2>,
                                      block_dual_large_kernel<8, false, 2>,  block_dual_large_kernel<9, false, 2>,
                                      block_dual_large_kernel<10, false, 2>, block_dual_large_kernel<11, false, 2>,
                                      block_dual_large_kernel<12, false, 2>, block_dual_large_kernel<13, false, 2>,
                                      block_dual_large_kernel<14, false, 2>, block_dual_large_kernel<15, false, 2>,
                                      block_dual_large_kernel<16, false, 2>};
  static const LargeKernel stack[] = {block_dual_large_kernel<1, true, 2>, block_dual_large_kernel<2, true, 2>,
                                      block_dual_large_kernel<3, true, 2>, block_dual_large_kernel<4, true, 2>,
                                      block_dual_large_kernel<5, true, 2>, block_dual_large_kernel<6, true, 2>,
                                      block_dual_large_kernel<7, true, 2>, block_dual_large_kernel<8, true, 2>};
  static const LargeKernel three[] = {block_dual_large_kernel<1, false, 3>, block_dual_large_kernel<2, false, 3>,
                                      block_dual_large_kernel<3, false, 3>, block_dual_large_kernel<4, false, 3>,
                                      block_dual_large_kernel<5, false, 3>, block_dual_large_kernel<6, false, 3>,
                                      block_dual_large_kernel<7, false, 3>, block_dual_large_kernel<8, false, 3>};
  if (parts == 3) return !stacked && k >= 1 && k <= kMaxStackedK ? three[k - 1] : nullptr;
  if (stacked) return k >= 1 && k <= kMaxStackedK ? stack[k - 1] : nullptr;
  return k >= kMinLargeK && k <= kMaxLargeK ? paper[k - kMinLargeK] : nullptr;
}
}  // namespace

cudaError_t block_dual_large_prepare(int k, bool stacked, size_t smem, int parts) {
  const LargeKernel f = large_kernel(k, stacked, parts);
  if (!f) return cudaErrorInvalidValue;
  int dev = 0, cap = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, f);
  if (e != cudaSuccess) return e;
  const size_t dyn = (size_t)cap > fa.sharedSizeBytes ? (size_t)cap - fa.sharedSizeBytes : 0;
  if (dyn < smem) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)dyn);
}

cudaError_t block_dual_large_occupancy(int k, bool stacked, size_t smem, int *ctas, int parts) {
  const LargeKernel f = large_kernel(k, stacked, parts);
  if (!f) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, f, block_dual_large_threads(k, stacked, parts), smem);
}

cudaError_t launch_block_dual_large(const BlockDualArgs &a, int k, bool stacked, int grid, size_t smem,
                                    cudaStream_t st, int parts) {
  const LargeKernel f = large_kernel(k, stacked, parts);
  if (!f) return cudaErrorInvalidValue;
  const size_t rows = block_dual_large_rows_floats(k, stacked, parts);
  if (rows && (!a.rows || rows * (size_t)grid > a.rows_cap)) return cudaErrorInvalidValue;
  f<<<grid, block_dual_large_threads(k, stacked, parts), smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace s3ttv
