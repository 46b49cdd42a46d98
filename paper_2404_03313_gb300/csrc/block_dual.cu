// Alg. 1 steps 8-11 for every block l (Sec. III-C):
//
//   Y'_l = Y_l + gamma_Y P_l D D_s ubar
//   Y_l  = Y'_l - gamma_Y prox_{gamma_Y^-1 ||.||_*}(Y'_l / gamma_Y)
//
// By Moreau's identity (eq. ProxConjugate) with eq. (prox_nuclear_norm) the second
// line clips the singular values of Y'_l at 1, independently of gamma_Y.  With
// G = Y' Y'^T (k^2 x k^2) = sum_x lam_x u_x u_x^T this is
//
//   Y_l = M Y'_l,   M = I - sum_{lam_x > 1} (1 - lam_x^-1/2) u_x u_x^T,
//
// so each block needs a k^2 x k^2 symmetric eigenproblem instead of an SVD of the
// k^2 x 2N3 block.  The kernel then scatters Z += P_l^T Y_l, the term step 2 of
// the next pass needs.
//
// Work decomposition: one CTA of kNW warps owns a group of kNW consecutive
// blocks at a time (a persistent grid strides over the groups).
//  1. For each block of the group in turn, its Y rows arrive in shared memory by
//     cp.async (the next block's rows are prefetched into L2 meanwhile) and
//     D D_s ubar (precomputed per pass as the cubes Fv, Fh) is added with weight
//     gamma_Y.  Rows are padded so the row stride is 4 mod 32 words and the
//     float4 reads of the Gram tiles do not conflict.
//  2. G = Y'Y'^T of that block: only tiles reaching the upper triangle are
//     formed (TR x K register tiles), the 2*N3 columns split across the warps,
//     partial tiles summed into the block's own G slot.
//  3. Warp w solves the eigenproblem of block w of the group by one-sided
//     (Hestenes) Jacobi on the rows of G: rotating pairs of rows until all rows
//     are mutually orthogonal leaves row x = lam_x u_x^T, so the eigenvalue is
//     the row norm and the eigenvector its direction; no rotation matrix is
//     accumulated.  Row pairs sit in lane pairs (each lane holds half of both
//     rows) and move between lanes in the odd-even order, so every pair of rows
//     meets once per sweep.  The kNW solves run side by side: one solve is a
//     chain of dependent shuffles and rotations, so an SM needs many of them in
//     flight to keep busy.
//  4. Warp w forms M = I - sum_x w_x u_x u_x^T of its block over that block's G
//     (stored by columns, in two halves).
//  5. For each block, Y' returns to shared memory (step 1 wrote it over Y_l in
//     global memory, where it stays in L2), every thread applies M to one float4
//     column chunk for half of the rows, in place; then the block's rows are
//     stored and added into Z (P_l^T Y_l) with float4 atomics.  Only one Y'
//     buffer is kept in shared memory, so four CTAs fit on an SM.
//
// Warm start: the rows of a block's eigenbasis change little from one pass of
// Alg. 1 to the next, so each block keeps its normalized converged rows W (one
// row per round-robin position) and the next pass starts the one-sided Jacobi
// from C0 = W G instead of G.  With W orthogonal, rows of J^T C0 that are
// mutually orthogonal are again lam_x u_x^T, so the result is the same
// decomposition; it only needs fewer sweeps.  A block whose rows did not all
// come out as nonzero directions stores a NaN marker and starts cold next time.
//
// First-order clip in the kept basis: when the stored rows W are still nearly
// an eigenbasis of this pass's G, the clip follows without any Jacobi sweep.
// B = W G W^T = D + O is then nearly diagonal, and the clip is the matrix
// function f(G) = W^T f(B) W with f(lam) = min(1, lam^-1/2).  To first order
// (the Daleckii-Krein expansion) f(B) = f(D) + F o O, F_ij the divided
// difference of f between d_i and d_j; the remainder is at most ||O||_F^2
// times half the largest |f''| near the spectrum, which stays finite as long as
// no eigenvalue can reach the kink at 1 (||O||_F < min_i |d_i - 1| / 4): 3/8
// lam_>^-5/2 above the kink (lam_> the smallest d_i above 1) plus, with d_i on
// both sides, 2 / min_i |d_i - 1| for a smooth bridge across it.  A block whose
// bound is within the fo_tol option takes M = W^T f(B) W (four 32 x 32 products
// on the tensor cores) and keeps its W; any other block runs the Jacobi, which
// stores fresh rows.  The divided differences are formed without cancellation:
// -1 / (sqrt(a) sqrt(b) (sqrt(a) + sqrt(b))) above the kink, and
// -(x - 1) / (sqrt(x) (1 + sqrt(x)) (x - y)) across it (x > 1 >= y).
#include <math.h>
#include "s3ttv_internal.cuh"

namespace s3ttv {
namespace {

constexpr int kNW = 4;  // warps per CTA

template <int K>
struct Shape {
  static constexpr int n = K * K;          // rows of a block (and of G)
  static constexpr int NP = (n + 1) / 2;   // row pairs (a zero row when n is odd)
  static constexpr int NPOS = 2 * NP;      // round-robin positions
  static constexpr int HP = (n + 3) / 4;   // column pairs of a row held by one lane
  static constexpr int HW = 2 * HP;        // columns held by one lane
  static constexpr int GS = (n + 2) & ~1;  // stride of G and of M (even)
  static constexpr int UTS = n;            // stride of the scaled eigen-rows
  static constexpr int TR = K < 3 ? K : 3; // Gram tile rows (tile columns: K)
  static constexpr int RH = (n + 1) / 2;   // rows per thread in the apply
  static constexpr int MH = (RH + 3) & ~3; // padded half of a column of M
  static constexpr int MS = (MH + n - RH + 3) & ~3;  // stride of the columns of M
  // Gram tiles: row groups of TR, column groups of K, those reaching the upper triangle
  static constexpr int NRG = (n + TR - 1) / TR;
  static constexpr int count_tiles() {
    int c = 0;
    for (int t = 0; t < NRG; ++t)
      for (int g = 0; g < K; ++g)
        if ((g + 1) * K - 1 >= t * TR) ++c;
    return c;
  }
  static constexpr int NT = count_tiles();
  static_assert(NT <= 32, "Gram tiles must fit one warp");
  static constexpr int TS = TR * K;        // entries per tile
};

// Tensor-core form: G and M padded to 32 x 32 and cut into 16 x 8 tiles
// (m-tile m: rows 16m..16m+15; n-tile q: columns 8q..8q+7).  The Gram needs
// the tiles that hold data and reach the upper triangle.
template <int K>
struct MmaShape {
  static constexpr int n = K * K;
  __host__ __device__ static constexpr bool need(int m, int q) { return 16 * m < n && 8 * q < n && 8 * q + 7 >= 16 * m; }
  static constexpr int count() {
    int c = 0;
    for (int m = 0; m < 2; ++m)
      for (int q = 0; q < 4; ++q)
        if (need(m, q)) ++c;
    return c;
  }
  static constexpr int NTILE = count();
  static constexpr int NM = (n + 15) / 16;  // m-tiles holding rows of M
  // The apply sums over the n rows of Y': full 8-row k-steps on tensor cores; a
  // remainder of one or two rows (n = 1, 9, 25) as FP32 FMAs, a longer one as
  // one more zero-padded k-step.
  static constexpr int NR0 = n % 8;
  static constexpr int NKS = n / 8 + (NR0 > 2 ? 1 : 0);  // tensor-core k-steps
  static constexpr int NR = NR0 > 2 ? 0 : NR0;           // rows left to FMAs
};

// One slot per block of the group: G, then the scaled eigen-rows (NPOS rows of
// stride UTS), then M.  CUDA-core form: M by columns in two halves; the float4
// reads of the last column's second half run MH floats past n * MS (values that
// multiply only unused rows).  Tensor-core form: M by rows, stride GS.
template <int K, bool TC>
__host__ __device__ constexpr int gm_floats() {
  using S = Shape<K>;
  constexpr int m = TC ? S::n * S::GS : S::n * S::MS + S::MH, u = S::NPOS * S::UTS, g = S::n * S::GS;
  constexpr int mu = m > u ? m : u;
  return ((mu > g ? mu : g) + 3) & ~3;
}

// Warm-start rows of one block: NPOS rows of n, padded to 16 bytes (the host's
// block_dual_w_stride).
template <int K>
__host__ __device__ constexpr int w_floats() {
  using S = Shape<K>;
  return (S::NPOS * S::n + 3) & ~3;
}

// Partial Gram tiles: CUDA-core form, every warp's register tiles; tensor-core
// form, the fragments of two warps (reduced in two rounds).
template <int K, bool TC>
__host__ __device__ constexpr int tiles_floats() {
  using S = Shape<K>;
  return TC ? 2 * MmaShape<K>::NTILE * 128 : (kNW * S::NT * S::TS + 3) & ~3;
}

// Scratch of the first-order clip, per warp: a NPOS x fo_stride matrix (C = W G,
// then f(B), then f(B) W) and a float4 per position (d, sqrt d, f(d), row of W
// present).  The stride is 4 mod 8 words, so the A-fragment reads (8 rows x 4
// consecutive words per access) hit 32 distinct banks.
template <int K>
__host__ __device__ constexpr int fo_stride() {
  return Shape<K>::NPOS + ((12 - Shape<K>::NPOS % 8) % 8);
}
template <int K>
__host__ __device__ constexpr int fo_floats() {
  return Shape<K>::NPOS * fo_stride<K>() + 4 * Shape<K>::NPOS;
}

// The Y' buffer: n rows of stride rs, also the staging area of the group's
// warm-start rows (and the first-order clip's scratch after them) during the
// eigen-solves and, in the tensor-core form, of the partial Gram tiles once the
// Gram has read Y'.
template <int K, bool TC>
__host__ __device__ constexpr size_t yp_floats(int rs) {
  const size_t y = (size_t)K * K * rs, w = (size_t)kNW * (w_floats<K>() + fo_floats<K>()),
               t = TC ? (size_t)tiles_floats<K, TC>() : 0;
  const size_t yw = y > w ? y : w;
  return yw > t ? yw : t;
}

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void sts4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// 16-byte global -> shared copy that bypasses L1 (cp.async, completes at wait_all)
__device__ __forceinline__ void cp_async16(float *sdst, const float *gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
// L2 eviction policies: the Y' rows written back after the Gram are kept
// (evict_last) until the apply reads them again, which marks them evict_first.
__device__ __forceinline__ unsigned long long l2_evict_last() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ unsigned long long l2_evict_first() {
  unsigned long long p;
  asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;\n" : "=l"(p));
  return p;
}
__device__ __forceinline__ void cp_async16_hint(float *sdst, const float *gsrc, unsigned long long pol) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global.L2::cache_hint [%0], [%1], 16, %2;\n" ::"r"(sa), "l"(gsrc), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void st_hint(float4 *p, float4 v, unsigned long long pol) {
  asm volatile("st.global.L2::cache_hint.v4.f32 [%0], {%1, %2, %3, %4}, %5;\n" ::"l"(p), "f"(v.x), "f"(v.y), "f"(v.z),
               "f"(v.w), "l"(pol)
               : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
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

// One warp: one-sided Jacobi on the rows of G (or of W G, Ws being a shared
// copy of the block's warm-start rows W, null for a cold start), then the
// scaled eigen-rows into Ut and the warm rows into W.  Returns the sweeps used.
// C0: the product W G already formed (rows of stride c0_ld), or null.
// wstage: shared memory of w_floats<K>() floats, free by the time the rows are
// final (it may be Ws or C0): the new W rows are assembled there and written
// out with coalesced 16-byte streaming stores; null: stored row by row.
template <int K>
__device__ int eigen_rows(const BlockDualArgs &a, long long l, const float *Ws, const float *Gm, float *Ut,
                          bool *ok, const float *C0 = nullptr, int c0_ld = 0, float *wstage = nullptr) {
  using S = Shape<K>;
  constexpr int n = S::n, NP = S::NP, NPOS = S::NPOS, HP = S::HP, HW = S::HW, GS = S::GS, UTS = S::UTS;
  const int lane = threadIdx.x & 31;
  // Positions 0..NPOS-1 hold the rows; lane pair i (lanes 2i, 2i+1, columns
  // [0, HW) and [HW, 2 HW) of both rows, as HP packed column pairs) holds
  // positions (2i, 2i+1) on even steps and (2i+1, 2i+2) on odd steps (the
  // odd-even ordering: neighbours rotate, then trade places, so every pair of
  // rows meets once in NPOS steps).  Between steps one row per lane moves one
  // lane pair along a ring; on odd steps the last lane pair holds (NPOS-1, 0),
  // which do not meet there.  Columns >= n stay 0.
  const int pi = lane >> 1, hf = lane & 1;
  const bool act = pi < NP;
  const int src_r = act ? (pi + 1 == NP ? hf : lane + 2) : lane;            // right neighbour (ring)
  const int src_l = act ? (pi == 0 ? 2 * (NP - 1) + hf : lane - 2) : lane;  // left neighbour (ring)
  const int col0 = hf * HW;
  // element (row r, column c) of a row-major matrix of stride ld, 0 outside
  auto ld2 = [&](const float *M, int ld, int r, bool ok_row, int c) -> f32x2 {
    const float x = (ok_row && c < n) ? M[r * ld + c] : 0.f;
    const float y = (ok_row && c + 1 < n) ? M[r * ld + c + 1] : 0.f;
    return pk2(x, y);
  };
  f32x2 A[HP], B[HP];
  const bool warm = Ws && !(Ws[0] != Ws[0]);  // NaN marks "start cold"
  if (warm && C0) {
#pragma unroll
    for (int j = 0; j < HP; ++j) {
      A[j] = ld2(C0, c0_ld, 2 * pi, act, col0 + 2 * j);
      B[j] = ld2(C0, c0_ld, 2 * pi + 1, act, col0 + 2 * j);
    }
  } else if (warm) {
    // C0 = W G: rows 2i, 2i+1 of W times G, this lane's columns
#pragma unroll
    for (int j = 0; j < HP; ++j) A[j] = B[j] = 0ull;
    const float *wra = Ws + (2 * pi) * n, *wrb = Ws + (2 * pi + 1) * n;
#pragma unroll 5
    for (int kk = 0; kk < n; ++kk) {
      const float wa = act ? wra[kk] : 0.f;
      const float wb = act ? wrb[kk] : 0.f;
      const f32x2 wa2 = pk2(wa, wa), wb2 = pk2(wb, wb);
#pragma unroll
      for (int j = 0; j < HP; ++j) {
        const f32x2 g = ld2(Gm, GS, kk, true, col0 + 2 * j);
        A[j] = fma2(wa2, g, A[j]);
        B[j] = fma2(wb2, g, B[j]);
      }
    }
  } else {
    const int rA = 2 * pi, rB = 2 * pi + 1;
#pragma unroll
    for (int j = 0; j < HP; ++j) {
      A[j] = ld2(Gm, GS, rA, act && rA < n, col0 + 2 * j);
      B[j] = ld2(Gm, GS, rB, act && rB < n, col0 + 2 * j);
    }
  }
  // squared row norms, tracked through the rotations and refreshed every sweep
  float nA, nB;
  auto refresh = [&]() {
    f32x2 x = 0ull, y = 0ull;
#pragma unroll
    for (int j = 0; j < HP; ++j) {
      x = fma2(A[j], A[j], x);
      y = fma2(B[j], B[j], y);
    }
    const float2 xs = up2(x), ys = up2(y);
    const float sa = xs.x + xs.y, sb = ys.x + ys.y;
    nA = sa + __shfl_xor_sync(kFull, sa, 1);
    nB = sb + __shfl_xor_sync(kFull, sb, 1);
  };
  refresh();
  float fro = hf == 0 ? nA + nB : 0.f;
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(kFull, fro, o);
  // Exact power-of-two scaling of the rows to a Frobenius norm near 1 keeps the
  // squares of the rotation parameters in range; eigenvalues are unscaled at
  // the end by inv_s.
  float inv_s = 1.f;
  if (fro > 0.f && fro < 1e30f) {
    const int ex = ((__float_as_int(fro) >> 23) & 255) - 127;  // fro = m 2^ex, m in [1, 2)
    const int h = ex >> 1;                                      // rows scale by 2^-h
    const float sc = __int_as_float((127 - h) << 23), sc2 = sc * sc;
    inv_s = __int_as_float((127 + h) << 23);
    const f32x2 scp = pk2(sc, sc);
#pragma unroll
    for (int j = 0; j < HP; ++j) {
      A[j] = mul2(A[j], scp);
      B[j] = mul2(B[j], scp);
    }
    nA *= sc2;
    nB *= sc2;
    fro *= sc2;
  }
  // rows below 1e-6 ||G||_F are numerical zeros: rotating them changes any
  // other row's direction by less than 1e-6
  const float floor2 = 1e-12f * fro;
  const float tol2 = a.tol * a.tol, pol2 = a.polish * a.polish;
  bool rotated = false;  // a pair less orthogonal than tol met in this sweep
  // One step.  The rows are rotated in place, A' = cA - sB, B' = sA + cB; read
  // with the positions of the odd-even ordering, A' now sits at B's position and
  // B' at A's (the pair traded places), so the movement below needs no copies.
  // The pair that does not meet on odd steps keeps its places, which in these
  // terms is the quarter turn (c, s) = (0, 1): its registers swap (one sign flips,
  // which changes nothing the solver uses).  When no pair of the warp needs a
  // rotation, meeting pairs are left as they are and only that swap remains.
  auto step = [&](bool meets, bool odd) {
    f32x2 p0 = 0ull, p1 = 0ull;  // two short chains
#pragma unroll
    for (int j = 0; j < HP; ++j) {
      if (j & 1) p1 = fma2(A[j], B[j], p1);
      else p0 = fma2(A[j], B[j], p0);
    }
    const float2 q0 = up2(p0), q1 = up2(p1);
    float apq = (q0.x + q0.y) + (q1.x + q1.y);
    apq += __shfl_xor_sync(kFull, apq, 1);
    const bool need = meets && fminf(nA, nB) > floor2 && apq * apq > pol2 * nA * nB;
    const bool quarter = act && !meets;  // the odd step's idle pair
    if (__any_sync(kFull, need)) {
      float c = quarter ? 0.f : 1.f, sn = quarter ? 1.f : 0.f, dn = 0.f;
      if (need) {
        // tan 2 theta = y / x with x = nB - nA, y = 2 apq and |theta| <= pi / 4:
        // cos 2 theta = |x| / r (r = |(x, y)|), c = sqrt((1 + cos 2 theta) / 2),
        // s = sign(x) y / (2 r c), t = s / c; two reciprocal square roots in all
        const float x = nB - nA, y = 2.f * apq;
        const float rr = rsqrtf(fmaf(x, x, y * y));
        const float hc = fmaf(0.5f * fabsf(x), rr, 0.5f);
        const float rc = rsqrtf(hc);
        c = hc * rc;
        sn = copysignf(0.5f, x) * y * rr * rc;
        dn = sn * rc * apq;  // t apq
        if (apq * apq > tol2 * nA * nB) rotated = true;
      }
      const f32x2 c2 = pk2(c, c), s2 = pk2(sn, sn), ns2 = pk2(-sn, -sn);
#pragma unroll
      for (int j = 0; j < HP; ++j) {
        const f32x2 x = A[j], y = B[j];
        A[j] = fma2(c2, x, mul2(ns2, y));
        B[j] = fma2(s2, x, mul2(c2, y));
      }
      const float oA = nA;
      nA = quarter ? nB : nA - dn;
      nB = quarter ? oA : nB + dn;
    } else if (odd) {
#pragma unroll
      for (int j = 0; j < HP; ++j) {
        const f32x2 x = A[j], y = B[j];
        A[j] = quarter ? y : x;
        B[j] = quarter ? x : y;
      }
      const float oA = nA;
      nA = quarter ? nB : nA;
      nB = quarter ? oA : nB;
    }
  };
  bool converged = false;
  int sweeps = 0;
  for (int sw = 0; sw < a.max_sweeps; ++sw) {
    rotated = false;
    if (sw) refresh();
#pragma unroll 1
    for (int sp = 0; sp < NPOS / 2; ++sp) {
      step(act, false);
      if constexpr (NP > 1) {  // to the odd positions: B takes the right neighbour's B
#pragma unroll
        for (int j = 0; j < HP; ++j) B[j] = __shfl_sync(kFull, B[j], src_r);
        nB = __shfl_sync(kFull, nB, src_r);
      }
      step(act && pi != NP - 1, true);
      if constexpr (NP > 1) {  // back to the even positions: A takes the left neighbour's A
#pragma unroll
        for (int j = 0; j < HP; ++j) A[j] = __shfl_sync(kFull, A[j], src_l);
        nA = __shfl_sync(kFull, nA, src_l);
      }
    }
    ++sweeps;
    if (!__any_sync(kFull, rotated)) {
      converged = true;
      break;
    }
  }
  *ok = converged;

  // eigen-rows: lam = ||row|| (unscaled), keep sqrt(1 - lam^-1/2) row / ||row||
  refresh();
  const float lA = sqrtf(nA) * inv_s, lB = sqrtf(nB) * inv_s;
  const float sA = lA > 1.f ? sqrtf(1.f - rsqrtf(lA)) * rsqrtf(nA) : 0.f;
  const float sB = lB > 1.f ? sqrtf(1.f - rsqrtf(lB)) * rsqrtf(nB) : 0.f;
  __syncwarp();  // Ut takes the place of G, which every lane has read
  if (act) {
#pragma unroll
    for (int j = 0; j < HP; ++j) {
      const float2 x = up2(A[j]), y = up2(B[j]);
      const int col = col0 + 2 * j;
      if (col < n) {
        Ut[(2 * pi) * UTS + col] = x.x * sA;
        Ut[(2 * pi + 1) * UTS + col] = y.x * sB;
      }
      if (col + 1 < n) {
        Ut[(2 * pi) * UTS + col + 1] = x.y * sA;
        Ut[(2 * pi + 1) * UTS + col + 1] = y.y * sB;
      }
    }
  }
  if (a.W) {
    // warm state for the next pass: the rows, normalized; all but the
    // NPOS - n zero rows must be nonzero directions, else mark the block cold
    const unsigned zero_rows = __popc(__ballot_sync(kFull, act && hf == 0 && nA <= floor2)) +
                               __popc(__ballot_sync(kFull, act && hf == 0 && nB <= floor2));
    float *Ww = a.W + (size_t)l * a.w_stride;
    if (zero_rows > (unsigned)(NPOS - n)) {
      if (lane == 0) Ww[0] = __int_as_float(0x7fc00000);
    } else {
      float *Wd = wstage ? wstage : Ww;
      if (act) {
        const float iA = nA > floor2 ? rsqrtf(nA) : 0.f, iB = nB > floor2 ? rsqrtf(nB) : 0.f;
#pragma unroll
        for (int j = 0; j < HP; ++j) {
          const float2 x = up2(A[j]), y = up2(B[j]);
          const int col = col0 + 2 * j;
          if (col < n) {
            Wd[(2 * pi) * n + col] = x.x * iA;
            Wd[(2 * pi + 1) * n + col] = y.x * iB;
          }
          if (col + 1 < n) {
            Wd[(2 * pi) * n + col + 1] = x.y * iA;
            Wd[(2 * pi + 1) * n + col + 1] = y.y * iB;
          }
        }
      }
      if (wstage) {
        __syncwarp();
        for (int c = lane; c < w_floats<K>() / 4; c += 32)
          __stcs(reinterpret_cast<float4 *>(Ww) + c, reinterpret_cast<const float4 *>(wstage)[c]);
        __syncwarp();  // wstage read before its next use
      }
    }
  }
  return sweeps;
}

// Warp w: M = I - Ut^T Ut of its own block, written over Ut (in the block's
// slot).  CUDA-core form: by columns, rows [0, RH) from slot 0 and rows [RH, n)
// from slot MH.  Tensor-core form: by rows, stride GS.
template <int K, bool TC>
__device__ void form_M(float *Gm) {
  const float *Ut = Gm;
  using S = Shape<K>;
  constexpr int n = S::n, GS = S::GS, RH = S::RH, MH = S::MH, MS = S::MS;
  const int lane = threadIdx.x & 31;
  const int R = lane / K, Sx = lane - R * K;
  float macc[K][K];
#pragma unroll
  for (int x = 0; x < K; ++x)
#pragma unroll
    for (int y = 0; y < K; ++y) macc[x][y] = 0.f;
  if (lane < n) {
#pragma unroll 2
    for (int xr = 0; xr < S::NPOS; ++xr) {
      float ua[K], ub[K];
#pragma unroll
      for (int x = 0; x < K; ++x) ua[x] = Ut[xr * S::UTS + R * K + x];
#pragma unroll
      for (int y = 0; y < K; ++y) ub[y] = Ut[xr * S::UTS + Sx * K + y];
#pragma unroll
      for (int x = 0; x < K; ++x)
#pragma unroll
        for (int y = 0; y < K; ++y) macc[x][y] = fmaf(ua[x], ub[y], macc[x][y]);
    }
  }
  __syncwarp();  // Ut no longer read
  if constexpr (TC) {
    if (lane < n) {
#pragma unroll
      for (int x = 0; x < K; ++x)
#pragma unroll
        for (int y = 0; y < K; ++y) {
          const int r = R * K + x, c = Sx * K + y;
          Gm[r * GS + c] = (r == c ? 1.f : 0.f) - macc[x][y];
        }
    }
  } else {
    for (int e = lane; e < n * MS; e += 32) Gm[e] = 0.f;
    __syncwarp();
    if (lane < n) {
#pragma unroll
      for (int x = 0; x < K; ++x)
#pragma unroll
        for (int y = 0; y < K; ++y) {
          const int r = R * K + x, c = Sx * K + y;
          const int slot = r < RH ? r : MH + (r - RH);
          Gm[c * MS + slot] = (r == c ? 1.f : 0.f) - macc[x][y];
        }
    }
  }
}

// d = A B for matrices of at most 32 x 32 on the tensor cores (one warp, three
// TF32 products per FP32 product): rows [0, MR) of A, columns [0, NC) of B and
// the inner index [0, KD) are read through the accessors, everything else is
// zero.  d[m][q][e] is element (16 m + g + 8 (e >> 1), 8 q + 2 t + (e & 1)) of
// the 32 x 32 result (g = lane / 4, t = lane % 4).
template <int MR, int NC, int KD, class FA, class FB>
__device__ __forceinline__ void mm32(const FA &A, const FB &B, float (&d)[2][4][4]) {
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q) d[m][q][0] = d[m][q][1] = d[m][q][2] = d[m][q][3] = 0.f;
#pragma unroll
  for (int kk = 0; kk < (KD + 7) / 8; ++kk) {
    unsigned bh[4][2], bl[4][2];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const int k = 8 * kk + t + 4 * h, j = 8 * q + g;
        split_tf32((8 * q < NC && k < KD && j < NC) ? B(k, j) : 0.f, bh[q][h], bl[q][h]);
      }
    unsigned ah[2][4], al[2][4];
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = 16 * m + g + 8 * (e & 1), k = 8 * kk + t + 4 * (e >> 1);
        split_tf32((16 * m < MR && i < MR && k < KD) ? A(i, k) : 0.f, ah[m][e], al[m][e]);
      }
    three_parts([&](auto P) {
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (16 * m < MR && 8 * q < NC)
            mma_3xtf32_part<decltype(P)::value>(d[m][q], ah[m], al[m], bh[q][0], bh[q][1], bl[q][0], bl[q][1]);
    });
  }
}

// Row and column of element e of result tile (m, q) for this lane.
__device__ __forceinline__ int frag_row(int m, int e) { return 16 * m + ((threadIdx.x & 31) >> 2) + 8 * (e >> 1); }
__device__ __forceinline__ int frag_col(int q, int e) { return 8 * q + 2 * (threadIdx.x & 3) + (e & 1); }

// Rows [0, MR) x columns [0, NC) of a result into a row-major matrix of stride ld.
template <int MR, int NC>
__device__ __forceinline__ void store_frag(const float (&d)[2][4][4], float *dst, int ld) {
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = frag_row(m, e), j = frag_col(q, e);
        if (i < MR && j < NC) dst[i * ld + j] = d[m][q][e];
      }
}

// M[r][c] = v into the block's M slot in the layout the apply reads: by rows of
// stride GS (tensor-core form) or by columns in two halves (CUDA-core form).
template <int K, bool TC>
__device__ __forceinline__ void put_M(float *Mg, int r, int c, float v) {
  using S = Shape<K>;
  if constexpr (TC) {
    Mg[r * S::GS + c] = v;
  } else {
    const int slot = r < S::RH ? r : S::MH + (r - S::RH);
    Mg[c * S::MS + slot] = v;
  }
}

// One warp: the first-order clip of its block in the kept basis (see the top
// of this file).  Ws: the block's stored rows W (NPOS rows of n; the padding
// position of an odd n holds zeros), Gm: G (stride GS), Sc / tab: this warp's
// scratch.  Returns true (warp-uniform) when the remainder bound is within
// fo_tol; then M has been written over Gm.  Returns false, with G untouched,
// otherwise.
template <int K, bool TC>
__device__ bool first_order_clip(const float *Ws, float *Gm, float *Sc, float4 *tab, float fo_tol) {
  using S = Shape<K>;
  constexpr int n = S::n, NPOS = S::NPOS, GS = S::GS, SS = fo_stride<K>();
  const int lane = threadIdx.x & 31;
  float d[2][4][4];
  // rows of W that hold a direction
  float wn = 0.f;
  if (lane < NPOS)
    for (int c = 0; c < n; ++c) wn = fmaf(Ws[lane * n + c], Ws[lane * n + c], wn);
  const unsigned present = __ballot_sync(kFull, lane < NPOS && wn > 0.5f);
  // C = W G, then B = C W^T
  mm32<NPOS, n, n>([&](int i, int k) { return Ws[i * n + k]; }, [&](int k, int j) { return Gm[k * GS + j]; }, d);
  store_frag<NPOS, n>(d, Sc, SS);
  __syncwarp();
  mm32<NPOS, NPOS, n>([&](int i, int k) { return Sc[i * SS + k]; }, [&](int k, int j) { return Ws[j * n + k]; },
                      d);
  float *tabf = reinterpret_cast<float *>(tab);
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = frag_row(m, e), j = frag_col(q, e);
        if (i == j && i < NPOS) tabf[4 * i] = d[m][q][e];
      }
  __syncwarp();
  // per position: d, sqrt d, f(d), present; the spectrum's distance to the kink
  const bool pr = (present >> lane) & 1u;
  float dmin = INFINITY, lgt = INFINITY;
  if (lane < NPOS) {
    const float dr = tabf[4 * lane];
    const float sr = sqrtf(fmaxf(dr, 0.f));
    const float fr = dr > 1.f ? rsqrtf(dr) : 1.f;
    tab[lane] = make_float4(dr, sr, fr, pr ? 1.f : 0.f);
    if (pr) {
      dmin = fabsf(dr - 1.f);
      if (dr > 1.f) lgt = dr;
    }
  }
  const unsigned above = __ballot_sync(kFull, pr && lgt < INFINITY);
  const unsigned below = present & ~above;
  // ||O||_F^2 over the present rows
  float os = 0.f;
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = frag_row(m, e), j = frag_col(q, e);
        if (i != j && i < NPOS && j < NPOS && ((present >> i) & (present >> j) & 1u)) os = fmaf(d[m][q][e], d[m][q][e], os);
      }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    os += __shfl_xor_sync(kFull, os, o);
    dmin = fminf(dmin, __shfl_xor_sync(kFull, dmin, o));
    lgt = fminf(lgt, __shfl_xor_sync(kFull, lgt, o));
  }
  float c = 0.f;
  if (above) {
    const float r = rsqrtf(lgt);
    c = 0.375f * r * r * r * r * r;
  }
  if (above && below) c += 2.f / dmin;
  const bool accept = present && sqrtf(os) < 0.25f * dmin && os * c <= fo_tol;
  if (!accept) return false;
  __syncwarp();  // the table is complete and every lane has read Gm
  if (!above) {
    // nothing clipped: f(B) = I on the present rows, so M = I
    if constexpr (!TC)
      for (int e = lane; e < n * S::MS; e += 32) Gm[e] = 0.f;
    __syncwarp();
    for (int e = lane; e < n * n; e += 32) {
      const int r = e / n, cc = e - r * n;
      put_M<K, TC>(Gm, r, cc, r == cc ? 1.f : 0.f);
    }
    return true;
  }
  // f(B): f(d_i) on the diagonal, divided differences times O off it
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = frag_row(m, e), j = frag_col(q, e);
        float x = 0.f;
        if (i < NPOS && j < NPOS && ((present >> i) & (present >> j) & 1u)) {
          const float4 ti = tab[i], tj = tab[j];
          if (i == j) {
            x = ti.z;
          } else {
            const bool hi = ti.x > 1.f, hj = tj.x > 1.f;
            float dd = 0.f;
            if (hi && hj) {
              dd = -__fdividef(ti.z * tj.z, ti.y + tj.y);
            } else if (hi || hj) {
              const float4 tx = hi ? ti : tj, ty = hi ? tj : ti;
              dd = -__fdividef((tx.x - 1.f) * tx.z, (1.f + tx.y) * (tx.x - ty.x));
            }
            x = dd * d[m][q][e];
          }
        }
        d[m][q][e] = x;
      }
  store_frag<NPOS, NPOS>(d, Sc, SS);
  __syncwarp();
  // T = f(B) W, then M = W^T T
  mm32<NPOS, n, NPOS>([&](int i, int k) { return Sc[i * SS + k]; }, [&](int k, int j) { return Ws[k * n + j]; },
                      d);
  __syncwarp();
  store_frag<NPOS, n>(d, Sc, SS);
  __syncwarp();
  mm32<n, n, NPOS>([&](int i, int k) { return Ws[k * n + i]; }, [&](int k, int j) { return Sc[k * SS + j]; }, d);
  if constexpr (!TC)
    for (int e = lane; e < n * S::MS; e += 32) Gm[e] = 0.f;
  __syncwarp();
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = frag_row(m, e), j = frag_col(q, e);
        if (i < n && j < n) put_M<K, TC>(Gm, i, j, d[m][q][e]);
      }
  return true;
}

// Tensor-core Gram of the block in Yp (n rows of stride RS, 2 N3p = 8 C4
// columns): warp w takes k-steps [w C4 / 4, (w+1) C4 / 4) of 8 columns, each
// operand split hi + lo; the four warps' partial tiles are summed in a fixed
// order (w0 + w2) + (w1 + w3) through Part (which may overlay Yp) and warp 0
// writes G (both triangles, each pair once, from the entry with i <= j).
// Called by all threads; holds barriers.
template <int K>
__device__ void gram_mma(const float *Yp, int RS, int C4, float *Part, float *Gb) {
  using T = MmaShape<K>;
  constexpr int n = T::n, GS = Shape<K>::GS, NTILE = T::NTILE;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float acc[NTILE][4];
#pragma unroll
  for (int i = 0; i < NTILE; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
  const int k0 = (C4 * warp) / kNW, k1 = (C4 * (warp + 1)) / kNW;
#pragma unroll 2
  for (int ks = k0; ks < k1; ++ks) {
    // x[q][h] = Y'[8q + g][8 ks + t + 4h], rows >= n read as 0
    unsigned xh[4][2], xl[4][2];
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        xh[q][h] = xl[q][h] = 0u;
        if (8 * q < n) {
          const int row = 8 * q + g;
          const float x = row < n ? Yp[(size_t)row * RS + 8 * ks + t + 4 * h] : 0.f;
          split_tf32(x, xh[q][h], xl[q][h]);
        }
      }
    const unsigned ah[2][4] = {{xh[0][0], xh[1][0], xh[0][1], xh[1][1]}, {xh[2][0], xh[3][0], xh[2][1], xh[3][1]}};
    const unsigned al[2][4] = {{xl[0][0], xl[1][0], xl[0][1], xl[1][1]}, {xl[2][0], xl[3][0], xl[2][1], xl[3][1]}};
    three_parts([&](auto P) {
      int idx = 0;
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (T::need(m, q)) {
            mma_3xtf32_part<decltype(P)::value>(acc[idx], ah[m], al[m], xh[q][0], xh[q][1], xl[q][0], xl[q][1]);
            ++idx;
          }
    });
  }
  float *P2 = Part, *P3 = Part + NTILE * 128;
  __syncthreads();  // the partials take the place of Y', which every warp has read
  if (warp >= 2) {
    float *P = warp == 2 ? P2 : P3;
#pragma unroll
    for (int i = 0; i < NTILE; ++i) sts4(P + i * 128 + lane * 4, make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]));
  }
  __syncthreads();
  if (warp < 2) {
    const float *P = warp == 0 ? P2 : P3;
#pragma unroll
    for (int i = 0; i < NTILE; ++i) {
      const float4 v = lds4(P + i * 128 + lane * 4);
      acc[i][0] += v.x;
      acc[i][1] += v.y;
      acc[i][2] += v.z;
      acc[i][3] += v.w;
    }
    if (warp == 1) {  // warp 1 alone read P3
#pragma unroll
      for (int i = 0; i < NTILE; ++i)
        sts4(P3 + i * 128 + lane * 4, make_float4(acc[i][0], acc[i][1], acc[i][2], acc[i][3]));
    }
  }
  __syncthreads();
  if (warp == 0) {
    int idx = 0;
#pragma unroll
    for (int m = 0; m < 2; ++m)
#pragma unroll
      for (int q = 0; q < 4; ++q)
        if (T::need(m, q)) {
          const float4 v = lds4(P3 + idx * 128 + lane * 4);
          const float d[4] = {acc[idx][0] + v.x, acc[idx][1] + v.y, acc[idx][2] + v.z, acc[idx][3] + v.w};
#pragma unroll
          for (int e = 0; e < 4; ++e) {
            const int i = 16 * m + g + 8 * (e >> 1), j = 8 * q + 2 * t + (e & 1);
            if (i < n && j < n && i <= j) {
              Gb[i * GS + j] = d[e];
              Gb[j * GS + i] = d[e];
            }
          }
          ++idx;
        }
  }
}

// Tensor-core apply, in place: Y'[s][c] (n rows of stride RS2, shared memory)
// becomes Y[r][c] = sum_s M[r][s] Y'[s][c].  Warp w takes the 8-column n-tiles
// [w C4 / 4, (w+1) C4 / 4) and reads, then writes, only those columns.  The A
// fragments of M (rows of stride GS) are split hi + lo into registers once; the
// B fragments of Y' one k-step at a time; the last NR rows of Y' are added with
// FP32 FMAs.
template <int K>
__device__ void apply_mma(float *Yp, int RS2, int C4, const float *Mg) {
  using T = MmaShape<K>;
  constexpr int n = T::n, GS = Shape<K>::GS, NM = T::NM, NKS = T::NKS, NR = T::NR, S0 = n - NR;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  const int q0 = (C4 * warp) / kNW, q1 = (C4 * (warp + 1)) / kNW;
  // A fragments of M: rows 16 m + g (+8), columns 8 kk + t (+4); columns >= S0
  // are the FMA rows, held as M[row][S0 + j]
  unsigned mh[NM][NKS > 0 ? NKS : 1][4], ml[NM][NKS > 0 ? NKS : 1][4];
  float mr[NM][2][NR > 0 ? NR : 1];
#pragma unroll
  for (int m = 0; m < NM; ++m) {
#pragma unroll
    for (int kk = 0; kk < NKS; ++kk)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int r = 16 * m + g + 8 * (e & 1), c = 8 * kk + t + 4 * (e >> 1);
        const float x = (r < n && c < S0) ? Mg[r * GS + c] : 0.f;
        split_tf32(x, mh[m][kk][e], ml[m][kk][e]);
      }
#pragma unroll
    for (int e2 = 0; e2 < 2; ++e2)
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const int r = 16 * m + g + 8 * e2;
        mr[m][e2][j] = r < n ? Mg[r * GS + S0 + j] : 0.f;
      }
  }
  // two n-tiles at a time: 2 NM independent accumulation chains per warp
#pragma unroll 1
  for (int q = q0; q < q1; q += 2) {
    const bool two = q + 1 < q1;
    float d[2][NM][4];
#pragma unroll
    for (int u = 0; u < 2; ++u)
#pragma unroll
      for (int m = 0; m < NM; ++m) d[u][m][0] = d[u][m][1] = d[u][m][2] = d[u][m][3] = 0.f;
#pragma unroll
    for (int kk = 0; kk < NKS; ++kk) {
      // B fragments: Y'[8 kk + t (+4)][8 (q + u) + g], rows >= S0 read as 0
      const int s0 = 8 * kk + t, s1 = s0 + 4;
      unsigned bh[2][2], bl[2][2];
#pragma unroll
      for (int u = 0; u < 2; ++u) {
        const float *col = Yp + 8 * (q + u) + g;
        const bool in = u == 0 || two;
        split_tf32(in && s0 < S0 ? col[(size_t)s0 * RS2] : 0.f, bh[u][0], bl[u][0]);
        split_tf32(in && s1 < S0 ? col[(size_t)s1 * RS2] : 0.f, bh[u][1], bl[u][1]);
      }
      three_parts([&](auto P) {
#pragma unroll
        for (int m = 0; m < NM; ++m)
#pragma unroll
          for (int u = 0; u < 2; ++u)
            mma_3xtf32_part<decltype(P)::value>(d[u][m], mh[m][kk], ml[m][kk], bh[u][0], bh[u][1], bl[u][0],
                                                bl[u][1]);
      });
    }
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && !two) break;
      // columns c, c + 1 of rows 16 m + g (+8)
      const int c = 8 * (q + u) + 2 * t;
#pragma unroll
      for (int j = 0; j < NR; ++j) {
        const float2 y = *reinterpret_cast<const float2 *>(Yp + (size_t)(S0 + j) * RS2 + c);
#pragma unroll
        for (int m = 0; m < NM; ++m)
#pragma unroll
          for (int e2 = 0; e2 < 2; ++e2) {
            d[u][m][2 * e2] = fmaf(mr[m][e2][j], y.x, d[u][m][2 * e2]);
            d[u][m][2 * e2 + 1] = fmaf(mr[m][e2][j], y.y, d[u][m][2 * e2 + 1]);
          }
      }
    }
    __syncwarp();  // every lane has read these columns
#pragma unroll
    for (int u = 0; u < 2; ++u) {
      if (u == 1 && !two) break;
      const int c = 8 * (q + u) + 2 * t;
#pragma unroll
      for (int m = 0; m < NM; ++m)
#pragma unroll
        for (int e2 = 0; e2 < 2; ++e2) {
          const int r = 16 * m + g + 8 * e2;
          if (r < n) *reinterpret_cast<float2 *>(Yp + (size_t)r * RS2 + c) = make_float2(d[u][m][2 * e2], d[u][m][2 * e2 + 1]);
        }
    }
  }
}

// This thread's share of a block's n x W4 grid of 16-byte chunks (rows r,
// chunks c4 of 4 floats): chunks c4 = c0, c0 + cs, ... < W4 and, for each,
// rows r = r0, r0 + rs, ... < n.  With W4 < threads, a thread keeps one chunk
// column (threads beyond the last whole set of columns stay idle), so the loops
// below carry no division.
// The steps cs, rs are the same for every thread.
struct Walk {
  int c0, r0;  // this thread's first chunk and row
  int cs, rs;  // steps
};
__device__ __forceinline__ Walk make_walk(int W4) {
  constexpr int NTH = kNW * 32;
  const int tid = threadIdx.x;
  Walk w;
  w.cs = W4 >= NTH ? NTH : W4;
  w.rs = W4 >= NTH ? 1 : NTH / W4;  // rows taken at once
  w.c0 = W4 >= NTH ? tid : tid % W4;
  w.r0 = W4 >= NTH ? 0 : tid / W4;
  if (w.r0 >= w.rs) w.c0 = W4;  // idle
  return w;
}

// Shared-memory copy of the n rows of Y_l (row stride RS); completes at
// cp_async_wait_all.
// With HINT the copies carry the L2 policy pol.
template <int K, bool HINT = false>
__device__ __forceinline__ void load_rows(float *Yp, const float *Yl, int RS, int N3p, int W4, const Walk &wk,
                                          unsigned long long pol = 0ull) {
  constexpr int n = K * K;
  for (int c4 = wk.c0; c4 < W4; c4 += wk.cs) {
    float *sp = Yp + (size_t)wk.r0 * RS + (c4 << 2);
    const float *gp = Yl + (size_t)wk.r0 * 2 * N3p + (c4 << 2);
    for (int r = wk.r0; r < n; r += wk.rs) {
      if constexpr (HINT) cp_async16_hint(sp, gp, pol);
      else cp_async16(sp, gp);
      sp += (size_t)wk.rs * RS;
      gp += (size_t)wk.rs * 2 * N3p;
    }
  }
}

// Start moving the n rows of Y_l (contiguous) into L2 ahead of their load.
template <int K>
__device__ __forceinline__ void prefetch_rows(const float *Yl, int N3p) {
  constexpr int n = K * K;
  const int lane = threadIdx.x & 31;
  for (int r = lane; r < n; r += 32)
    asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(Yl + (size_t)r * 2 * N3p),
                 "r"((unsigned)(2 * N3p * sizeof(float)))
                 : "memory");
}

// MINB: CTAs per SM the register budget is sized for (5: 96 registers a thread,
// 4: 128), the largest whose shared memory fits on an SM.
// TC: Gram and apply on tensor cores (three TF32 products per FP32 product)
// instead of FP32 CUDA cores.
template <int K, int MINB, bool TC>
__global__ void __launch_bounds__(kNW * 32, MINB) block_dual_kernel(BlockDualArgs a) {
  using S = Shape<K>;
  constexpr int n = S::n, GS = S::GS, TR = S::TR, NT = S::NT, TS = S::TS, RH = S::RH, MH = S::MH,
                MS = S::MS;
  constexpr int NTH = kNW * 32;
  constexpr int NF = 6;  // F loads in flight per thread
  extern __shared__ __align__(16) float smem[];
  __shared__ unsigned s_sweeps, s_fo;
  __shared__ int s_tile_r0[TC ? 1 : 32], s_tile_c0[TC ? 1 : 32];
  __shared__ int s_off[kNW][n];  // pixel (i * N2 + j) of row r of P_l
  __shared__ int s_queued[kNW];  // block b of the group went to the FP64 re-solve
  if (a.sc->done) return;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int RS = a.rs;                              // row stride of the block copies
  float *Yp = smem;                                 // Y' (then Y) of one block
  float *Gall = Yp + yp_floats<K, TC>(RS);          // kNW x (G, eigen-rows, M)
  float *Tiles = TC ? Yp : Gall + kNW * gm_floats<K, TC>();  // partial Gram tiles
  const Dims dm = a.dm;
  const int N3p = dm.N3p, C4 = N3p >> 2, W4 = 2 * C4;
  const long long L = dm.P;
  const long long groups = (L + kNW - 1) / kNW;
  const float gY = a.gY;
  const bool warm = a.warm && a.W;  // a.w_stride == w_floats<K>()
  const Walk wk = make_walk(W4);
  const unsigned long long pol_keep = l2_evict_last(), pol_done = l2_evict_first();
  if (tid == 0 && !TC) {
    int c = 0;
    for (int t = 0; t < S::NRG; ++t)
      for (int g = 0; g < K; ++g)
        if ((g + 1) * K - 1 >= t * TR) {
          s_tile_r0[c] = t * TR;
          s_tile_c0[c] = g * K;
          ++c;
        }
  }
  if (tid == 0) s_sweeps = s_fo = 0u;
  __syncthreads();

  for (long long grp = blockIdx.x; grp < groups; grp += gridDim.x) {
    const long long l0 = grp * kNW;
    const int nb = (int)(L - l0 < kNW ? L - l0 : kNW);  // blocks in this group
    if (warm && warp == 2 && lane < nb)  // warm-start rows into L2 for step 3
      asm volatile("cp.async.bulk.prefetch.L2.global [%0], %1;\n" ::"l"(a.W + (size_t)(l0 + lane) * w_floats<K>()),
                   "r"((unsigned)(w_floats<K>() * sizeof(float)))
                   : "memory");

    // ---- 1-2. for each block of the group: Y' in shared memory, then its Gram ----
    for (int b = 0; b < nb; ++b) {
      const long long l = l0 + b;
      float *Yl = a.Y + (size_t)l * n * 2 * N3p;
      load_rows<K, true>(Yp, Yl, RS, N3p, W4, wk, pol_done);
      if (warp == 1 && b + 1 < nb) prefetch_rows<K>(Yl + (size_t)n * 2 * N3p, N3p);
      if (tid < n) {
        const int p = (int)(l / dm.N2), q = (int)(l - (long long)p * dm.N2);
        const int ra = tid / K, rc = tid - ra * K;
        int i = p + ra;
        if (i >= dm.N1) i -= dm.N1;
        int j = q + rc;
        if (j >= dm.N2) j -= dm.N2;
        s_off[b][tid] = i * dm.N2 + j;
      }
      cp_async_wait_all();
      __syncthreads();
      // Y' = Y + gamma_Y (Fv | Fh), NF loads of D D_s ubar in flight per thread
      for (int c4 = wk.c0; c4 < W4; c4 += wk.cs) {
        const bool hz = c4 >= C4;
        const float *Fb = (hz ? a.Fh : a.Fv) + ((hz ? c4 - C4 : c4) << 2);
        for (int rb = wk.r0; rb < n; rb += NF * wk.rs) {
          float4 xv[NF];
#pragma unroll
          for (int u = 0; u < NF; ++u) {
            const int r = rb + u * wk.rs;
            if (r < n) xv[u] = __ldg(reinterpret_cast<const float4 *>(Fb + (size_t)s_off[b][r] * N3p));
          }
#pragma unroll
          for (int u = 0; u < NF; ++u) {
            const int r = rb + u * wk.rs;
            if (r < n) {
              float *dst = Yp + (size_t)r * RS + (c4 << 2);
              float4 y = lds4(dst);
              y.x = fmaf(gY, xv[u].x, y.x);
              y.y = fmaf(gY, xv[u].y, y.y);
              y.z = fmaf(gY, xv[u].z, y.z);
              y.w = fmaf(gY, xv[u].w, y.w);
              sts4(dst, y);
              // Y' replaces Y_l in global memory (kept in L2) for step 5
              st_hint(reinterpret_cast<float4 *>(Yl + (size_t)r * 2 * N3p) + c4, y, pol_keep);
            }
          }
        }
      }
      __syncthreads();
      if constexpr (TC) {
        gram_mma<K>(Yp, RS, C4, Tiles, Gall + b * gm_floats<K, TC>());
      } else {
        if (lane < NT) {  // tiles reaching the upper triangle, this warp's share of the columns
          const int r0 = s_tile_r0[lane], c0 = s_tile_c0[lane];
          float acc[TR][K];
#pragma unroll
          for (int x = 0; x < TR; ++x)
#pragma unroll
            for (int y = 0; y < K; ++y) acc[x][y] = 0.f;
          const float *pa = Yp + (size_t)r0 * RS;
          const float *pb = Yp + (size_t)c0 * RS;
          const int q0 = (W4 * warp) / kNW, q1 = (W4 * (warp + 1)) / kNW;
#pragma unroll 2
          for (int qq = q0; qq < q1; ++qq) {
            const int c = qq << 2;
            float4 va[TR], vb[K];
#pragma unroll
            for (int x = 0; x < TR; ++x)
              va[x] = (r0 + x < n) ? lds4(pa + (size_t)x * RS + c) : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
            for (int y = 0; y < K; ++y) vb[y] = lds4(pb + (size_t)y * RS + c);
#pragma unroll
            for (int x = 0; x < TR; ++x)
#pragma unroll
              for (int y = 0; y < K; ++y) {
                float t = acc[x][y];
                t = fmaf(va[x].x, vb[y].x, t);
                t = fmaf(va[x].y, vb[y].y, t);
                t = fmaf(va[x].z, vb[y].z, t);
                t = fmaf(va[x].w, vb[y].w, t);
                acc[x][y] = t;
              }
          }
          float *pt = Tiles + ((size_t)warp * NT + lane) * TS;
#pragma unroll
          for (int x = 0; x < TR; ++x)
#pragma unroll
            for (int y = 0; y < K; ++y) pt[x * K + y] = acc[x][y];
        }
        __syncthreads();
        float *Gb = Gall + b * gm_floats<K, TC>();
        for (int e = tid; e < NT * TS; e += NTH) {
          const int tl = e / TS, w = e - tl * TS, x = w / K, y = w - x * K;
          const int r = s_tile_r0[tl] + x, c = s_tile_c0[tl] + y;
          if (r < n) {
            float g = 0.f;
#pragma unroll
            for (int ww = 0; ww < kNW; ++ww) g += Tiles[((size_t)ww * NT + tl) * TS + w];
            Gb[r * GS + c] = g;
            Gb[c * GS + r] = g;
          }
        }
      }
      __syncthreads();
    }

    // ---- 3-4. every warp: eigen-solve of one block of the group, then its M ----
    if (warp == 0 && grp + gridDim.x < groups)  // the next group's first block
      prefetch_rows<K>(a.Y + (size_t)(grp + gridDim.x) * kNW * n * 2 * N3p, N3p);
    if (warm) {  // the group's warm-start rows into the free Y' buffer
      constexpr int WS4 = w_floats<K>() / 4;
      for (int idx = tid; idx < nb * WS4; idx += NTH) {
        const int b = idx / WS4, c = idx - b * WS4;
        cp_async16(Yp + b * w_floats<K>() + 4 * c, a.W + (size_t)(l0 + b) * w_floats<K>() + 4 * c);
      }
      cp_async_wait_all();
      __syncthreads();
    }
    if (warp < nb) {
      float *Gb = Gall + warp * gm_floats<K, TC>();
      const float *Ws = warm ? Yp + warp * w_floats<K>() : nullptr;
      bool fo = false;
      const float *C0 = nullptr;  // W G, formed by a first-order attempt that fell through
      if (Ws && a.fo_tol > 0.f && !(Ws[0] != Ws[0])) {
        float *Sc = Yp + kNW * w_floats<K>() + warp * fo_floats<K>();
        fo = first_order_clip<K, TC>(Ws, Gb, Sc, reinterpret_cast<float4 *>(Sc + S::NPOS * fo_stride<K>()),
                                     a.fo_tol);
        C0 = Sc;
      }
      if (fo) {
        if (lane == 0) {
          s_queued[warp] = 0;
          atomicAdd(&s_fo, 1u);
        }
        __syncwarp();
      } else {
      bool ok;
      const int sweeps = eigen_rows<K>(a, l0 + warp, Ws, Gb, Gb, &ok, C0, fo_stride<K>());
      if (lane == 0) {
        int queued = 0;
        if (!ok) {
          // to the FP64 re-solve if the queue has room; else applied as it stands
          const unsigned slot = a.fb_list ? atomicAdd(&a.sc->fb_count, 1u) : 0xffffffffu;
          if (slot < (unsigned)a.fb_cap) {
            a.fb_list[slot] = (int)(l0 + warp);
            queued = 1;
          } else {
            atomicAdd(&a.sc->jacobi_fail, 1u);
          }
        }
        s_queued[warp] = queued;
        atomicAdd(&s_sweeps, (unsigned)sweeps);
      }
      __syncwarp();
      form_M<K, TC>(Gb);
      }
    }
    __syncthreads();

    // ---- 5. for each block: Y' back into shared memory, Y_l = M Y' in place, then
    //         Y_l stored and P_l^T Y_l added into Z, row by row ----
    for (int b = 0; b < nb; ++b) {
      if (s_queued[b]) continue;  // CTA-uniform: Y_l keeps Y' for the FP64 re-solve
      const long long l = l0 + b;
      float *Yl = a.Y + (size_t)l * n * 2 * N3p;
      const float *Mg = Gall + b * gm_floats<K, TC>();
      load_rows<K, true>(Yp, Yl, RS, N3p, W4, wk, pol_done);
      cp_async_wait_all();
      __syncthreads();
      if constexpr (TC) {
        apply_mma<K>(Yp, RS, C4, Mg);
      } else {
        // task: one float4 column chunk, half of the rows.  The two tasks of a chunk
        // are neighbouring lanes of one warp in the same round, so a warp barrier
        // orders every read of the chunk before it is overwritten with Y_l.
        for (int base = 0; base < 2 * W4; base += NTH) {
          const int task = base + tid;
          const bool has = task < 2 * W4;
          const int c4 = task >> 1, half = task & 1;
          float4 acc[RH];
#pragma unroll
          for (int x = 0; x < RH; ++x) acc[x] = make_float4(0.f, 0.f, 0.f, 0.f);
          if (has) {
            const float *col = Yp + (c4 << 2);
#pragma unroll(MINB >= 5 ? 1 : 5)
            for (int s = 0; s < n; ++s) {
              const float4 y = lds4(col + (size_t)s * RS);
              const float *mcol = Mg + s * MS + half * MH;  // M[r][s] for this half's rows
#pragma unroll
              for (int x4 = 0; x4 < MH; x4 += 4) {
                const float4 m = lds4(mcol + x4);
                const float mm[4] = {m.x, m.y, m.z, m.w};
#pragma unroll
                for (int e = 0; e < 4; ++e) {
                  if (x4 + e < RH) {
                    acc[x4 + e].x = fmaf(mm[e], y.x, acc[x4 + e].x);
                    acc[x4 + e].y = fmaf(mm[e], y.y, acc[x4 + e].y);
                    acc[x4 + e].z = fmaf(mm[e], y.z, acc[x4 + e].z);
                    acc[x4 + e].w = fmaf(mm[e], y.w, acc[x4 + e].w);
                  }
                }
              }
            }
          }
          __syncwarp();
          if (has) {
            float *dst = Yp + (size_t)(half * RH) * RS + (c4 << 2);
#pragma unroll
            for (int x = 0; x < RH; ++x)
              if (half * RH + x < n) sts4(dst + (size_t)x * RS, acc[x]);
          }
        }
      }
      __syncthreads();  // Y_l complete in shared memory
      for (int c4 = wk.c0; c4 < W4; c4 += wk.cs) {
        const bool hz = c4 >= C4;
        float *Zb = (hz ? a.Zh : a.Zv) + ((hz ? c4 - C4 : c4) << 2);
        for (int r = wk.r0; r < n; r += wk.rs) {
          const float4 y = lds4(Yp + (size_t)r * RS + (c4 << 2));
          __stcs(reinterpret_cast<float4 *>(Yl + (size_t)r * 2 * N3p) + c4, y);
          atomicAdd(reinterpret_cast<float4 *>(Zb + (size_t)s_off[b][r] * N3p), y);
        }
      }
      __syncthreads();  // the shared buffer is free for the next block
    }
  }
  if (tid == 0 && s_sweeps) atomicAdd(&a.sc->jacobi_sweeps, (unsigned long long)s_sweeps);
  if (tid == 0 && s_fo) atomicAdd(&a.sc->fo_blocks, (unsigned long long)s_fo);
}

// One warp: M = I - Ut^T Ut of its block on the tensor cores, written over Ut
// by rows of stride GS (Ut: NPOS rows of stride UTS = n in the block's slot).
template <int K>
__device__ void form_M_mma(float *Gm) {
  using S = Shape<K>;
  constexpr int n = S::n, NPOS = S::NPOS, GS = S::GS;
  float d[2][4][4];
  mm32<n, n, NPOS>([&](int i, int k) { return Gm[k * S::UTS + i]; },
                   [&](int k, int j) { return Gm[k * S::UTS + j]; }, d);
  __syncwarp();  // Ut no longer read
#pragma unroll
  for (int m = 0; m < 2; ++m)
#pragma unroll
    for (int q = 0; q < 4; ++q)
#pragma unroll
      for (int e = 0; e < 4; ++e) {
        const int i = frag_row(m, e), j = frag_col(q, e);
        if (i < n && j < n) Gm[i * GS + j] = (i == j ? 1.f : 0.f) - d[m][q][e];
      }
}

// ---------------------------------------------------------------------------
// Streaming form (k <= 5, tensor cores): every warp owns one block at a time,
// end to end, and streams its rows through two chunk buffers of kCW columns,
// so the copies of the next chunk are in flight while the current one is
// used, and no step waits on a CTA-wide barrier.
//  A. For each chunk: Y rows by cp.async (the next chunk's issued first),
//     Y' = Y + gamma_Y (Fv | Fh), written back over Y_l, and the chunk's part
//     of G = Y'Y'^T on the tensor cores (the warp holds all of G in registers).
//  B. The clip of the block: first-order in the kept basis, else the Jacobi
//     (the same device code as the group form above), M over G's slot.
//  C. For each chunk: Y' back from global memory, Y_l = M Y' in place, Y_l
//     stored and P_l^T Y_l added into Z.
// While a warp is in B its chunk buffers hold the block's stored rows W and
// the first-order scratch.
constexpr int kSW = 4;         // warps per CTA
constexpr int kCW = 32;        // columns per chunk (four 8-column k-steps)
constexpr int kCS = kCW + 4;   // chunk row stride: 4 mod 32 words (conflict-free Gram fragments)

template <int K>
struct StreamLayout {
  static constexpr int n = K * K;
  static constexpr int buf = n * kCS;                          // one chunk buffer
  static constexpr int gm = gm_floats<K, true>();              // G, then M (by rows, stride GS)
  static constexpr int off = 2 * buf + gm;                     // the rows' pixel offsets (n ints)
  static constexpr int fb = (off + n + 3) & ~3;                // the chunk's F rows (n x kCW), step A
  static constexpr int per_warp = fb + n * kCW;
  static_assert(w_floats<K>() + fo_floats<K>() <= 2 * buf, "W and the first-order scratch fit the chunk buffers");
};

__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N>
__device__ __forceinline__ void cp_async_wait() {
  asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// One block l of the problem a, by the calling warp (see above).  bufs: the
// warp's shared region (two chunk buffers, then G / M, then the rows' pixel
// offsets, laid out for K); the statistics go to sweeps and fo_count.
template <int K>
__device__ void stream_block(const BlockDualArgs &a, long long l, float *bufs, unsigned long long pol_keep,
                             unsigned long long pol_done, unsigned long long &sweeps,
                             unsigned long long &fo_count) {
  using S = Shape<K>;
  using T = MmaShape<K>;
  using LY = StreamLayout<K>;
  constexpr int n = S::n, GS = S::GS, NTILE = T::NTILE, NM = T::NM, NKS = T::NKS, NR = T::NR, S0 = n - NR;
  constexpr int NE = (n * (kCW / 4) + 31) / 32;  // 16-byte pieces of a chunk per lane
  const int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3;
  float *Gm = bufs + 2 * LY::buf;
  int *off = reinterpret_cast<int *>(bufs + LY::off);
  float *fb = bufs + LY::fb;
  const Dims dm = a.dm;
  const int N3p = dm.N3p, RW = 2 * N3p, NCH = (RW + kCW - 1) / kCW;
  const float gY = a.gY;
  const bool warm = a.warm && a.W;  // a.w_stride == w_floats<K>()
  {
    float *Yl = a.Y + (size_t)l * n * RW;
    if (lane < n) {
      const int p = (int)(l / dm.N2), q = (int)(l - (long long)p * dm.N2);
      const int ra = lane / K, rc = lane - ra * K;
      int i = p + ra;
      if (i >= dm.N1) i -= dm.N1;
      int j = q + rc;
      if (j >= dm.N2) j -= dm.N2;
      off[lane] = i * dm.N2 + j;
    }
    // chunk ch of the n rows into buffer b: piece e = (row e / 8, float4 e % 8)
    auto load_chunk = [&](int ch, float *b, unsigned long long pol) {
      const int c0 = ch * kCW, w4 = min(kCW, RW - c0) >> 2;
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        const int e = lane + 32 * u, r = e >> 3, j = e & 7;
        if (r < n && j < w4) cp_async16_hint(b + r * kCS + 4 * j, Yl + (size_t)r * RW + c0 + 4 * j, pol);
      }
      cp_async_commit();
    };
    // the F rows of chunk ch (F = (Fv | Fh) at the rows' pixels) into fb, the
    // same pieces as load_chunk; its own commit group
    auto load_f = [&](int ch) {
      const int c0 = ch * kCW, w4 = min(kCW, RW - c0) >> 2;
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        const int e = lane + 32 * u, r = e >> 3, j = e & 7;
        if (r < n && j < w4) {
          const int c = c0 + 4 * j;
          const bool hz = c >= N3p;
          cp_async16(fb + r * kCW + 4 * j, (hz ? a.Fh : a.Fv) + (size_t)off[r] * N3p + (hz ? c - N3p : c));
        }
      }
      cp_async_commit();
    };
    __syncwarp();  // the pixel offsets are visible; the buffers are free

    // ---- A. Y' chunk by chunk, its Gram in registers ----
    float acc[NTILE][4];
#pragma unroll
    for (int i = 0; i < NTILE; ++i) acc[i][0] = acc[i][1] = acc[i][2] = acc[i][3] = 0.f;
    // Commit groups in order: Y(0), F(0), then per chunk ch: Y(ch + 1) before
    // the wait, F(ch + 1) once F(ch) has been used, so waiting for all but the
    // newest group leaves Y(ch) and F(ch) complete.
    load_chunk(0, bufs, pol_done);
    load_f(0);
    for (int ch = 0; ch < NCH; ++ch) {
      float *cur = bufs + (ch & 1) * LY::buf;
      if (ch + 1 < NCH) {
        load_chunk(ch + 1, bufs + ((ch + 1) & 1) * LY::buf, pol_done);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      const int c0 = ch * kCW, w4 = min(kCW, RW - c0) >> 2;
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        const int e = lane + 32 * u, r = e >> 3, j = e & 7;
        if (r < n && j < w4) {
          float *dst = cur + r * kCS + 4 * j;
          const float4 f = lds4(fb + r * kCW + 4 * j);
          float4 y = lds4(dst);
          y.x = fmaf(gY, f.x, y.x);
          y.y = fmaf(gY, f.y, y.y);
          y.z = fmaf(gY, f.z, y.z);
          y.w = fmaf(gY, f.w, y.w);
          sts4(dst, y);
          // Y' replaces Y_l in global memory (kept in L2) for step C
          st_hint(reinterpret_cast<float4 *>(Yl + (size_t)r * RW + c0) + j, y, pol_keep);
        }
      }
      __syncwarp();  // every lane has read fb: the next chunk's F may replace it
      if (ch + 1 < NCH) load_f(ch + 1);
      const int nks = w4 >> 1;
      for (int ks = 0; ks < nks; ++ks) {
        unsigned xh[4][2], xl[4][2];
#pragma unroll
        for (int q = 0; q < 4; ++q)
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            xh[q][h] = xl[q][h] = 0u;
            if (8 * q < n) {
              const int row = 8 * q + g;
              split_tf32(row < n ? cur[row * kCS + 8 * ks + t + 4 * h] : 0.f, xh[q][h], xl[q][h]);
            }
          }
        const unsigned ah[2][4] = {{xh[0][0], xh[1][0], xh[0][1], xh[1][1]}, {xh[2][0], xh[3][0], xh[2][1], xh[3][1]}};
        const unsigned al[2][4] = {{xl[0][0], xl[1][0], xl[0][1], xl[1][1]}, {xl[2][0], xl[3][0], xl[2][1], xl[3][1]}};
        three_parts([&](auto P) {
          int idx = 0;
#pragma unroll
          for (int m = 0; m < 2; ++m)
#pragma unroll
            for (int q = 0; q < 4; ++q)
              if (T::need(m, q)) {
                mma_3xtf32_part<decltype(P)::value>(acc[idx], ah[m], al[m], xh[q][0], xh[q][1], xl[q][0], xl[q][1]);
                ++idx;
              }
        });
      }
      __syncwarp();  // every lane has read this buffer before it is refilled
    }
    {  // G, both triangles, from the tiles reaching the upper triangle
      int idx = 0;
#pragma unroll
      for (int m = 0; m < 2; ++m)
#pragma unroll
        for (int q = 0; q < 4; ++q)
          if (T::need(m, q)) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              const int i = 16 * m + g + 8 * (e >> 1), j = 8 * q + 2 * t + (e & 1);
              if (i < n && j < n && i <= j) {
                Gm[i * GS + j] = acc[idx][e];
                Gm[j * GS + i] = acc[idx][e];
              }
            }
            ++idx;
          }
    }

    // ---- B. the clip: M over G's slot ----
    const float *Ws = nullptr;
    if (warm) {  // the block's stored rows into the (now idle) chunk buffers
      const float *Wg = a.W + (size_t)l * w_floats<K>();
      for (int c = lane; c < w_floats<K>() / 4; c += 32) cp_async16(bufs + 4 * c, Wg + 4 * c);
      cp_async_commit();
      cp_async_wait<0>();
      Ws = bufs;
    }
    __syncwarp();  // G and W visible to every lane
    bool fo = false;
    const float *C0 = nullptr;  // the warm-start product W G, on the tensor cores
    if (Ws && !(Ws[0] != Ws[0])) {
      float *Sc = bufs + w_floats<K>();
      if (a.fo_tol > 0.f) {
        fo = first_order_clip<K, true>(Ws, Gm, Sc, reinterpret_cast<float4 *>(Sc + S::NPOS * fo_stride<K>()),
                                       a.fo_tol);
      } else {
        float d[2][4][4];
        mm32<S::NPOS, n, n>([&](int i, int k) { return Ws[i * n + k]; },
                            [&](int k, int j) { return Gm[k * GS + j]; }, d);
        store_frag<S::NPOS, n>(d, Sc, fo_stride<K>());
        __syncwarp();
      }
      C0 = Sc;
    }
    if (fo) {
      ++fo_count;
    } else {
      bool ok;
      sweeps += eigen_rows<K>(a, l, Ws, Gm, Gm, &ok, C0, fo_stride<K>(), bufs);
      int queued = 0;
      if (lane == 0 && !ok) {
        // to the FP64 re-solve if the queue has room; else applied as it stands
        const unsigned slot = a.fb_list ? atomicAdd(&a.sc->fb_count, 1u) : 0xffffffffu;
        if (slot < (unsigned)a.fb_cap) {
          a.fb_list[slot] = (int)l;
          queued = 1;
        } else {
          atomicAdd(&a.sc->jacobi_fail, 1u);
        }
      }
      queued = __shfl_sync(kFull, queued, 0);
      __syncwarp();
      form_M_mma<K>(Gm);
      if (queued) return;  // Y_l keeps Y' for the FP64 re-solve, nothing added to Z
    }
    __syncwarp();  // M visible to every lane; W and the scratch are no longer read

    // ---- C. Y_l = M Y' chunk by chunk, stored and added into Z ----
    unsigned mh[NM][NKS > 0 ? NKS : 1][4], ml[NM][NKS > 0 ? NKS : 1][4];
    float mr[NM][2][NR > 0 ? NR : 1];
#pragma unroll
    for (int m = 0; m < NM; ++m) {
#pragma unroll
      for (int kk = 0; kk < NKS; ++kk)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int r = 16 * m + g + 8 * (e & 1), c = 8 * kk + t + 4 * (e >> 1);
          split_tf32((r < n && c < S0) ? Gm[r * GS + c] : 0.f, mh[m][kk][e], ml[m][kk][e]);
        }
#pragma unroll
      for (int e2 = 0; e2 < 2; ++e2)
#pragma unroll
        for (int j = 0; j < NR; ++j) {
          const int r = 16 * m + g + 8 * e2;
          mr[m][e2][j] = r < n ? Gm[r * GS + S0 + j] : 0.f;
        }
    }
    load_chunk(0, bufs, pol_done);
    for (int ch = 0; ch < NCH; ++ch) {
      float *cur = bufs + (ch & 1) * LY::buf;
      if (ch + 1 < NCH) {
        load_chunk(ch + 1, bufs + ((ch + 1) & 1) * LY::buf, pol_done);
        cp_async_wait<1>();
      } else {
        cp_async_wait<0>();
      }
      __syncwarp();
      const int c0 = ch * kCW, w4 = min(kCW, RW - c0) >> 2, ntl = w4 >> 1;
      // n-tiles of 8 columns, two at a time
      for (int q = 0; q < ntl; q += 2) {
        const bool two = q + 1 < ntl;
        float d[2][NM][4];
#pragma unroll
        for (int u = 0; u < 2; ++u)
#pragma unroll
          for (int m = 0; m < NM; ++m) d[u][m][0] = d[u][m][1] = d[u][m][2] = d[u][m][3] = 0.f;
#pragma unroll
        for (int kk = 0; kk < NKS; ++kk) {
          const int s0 = 8 * kk + t, s1 = s0 + 4;
          unsigned bh[2][2], bl[2][2];
#pragma unroll
          for (int u = 0; u < 2; ++u) {
            const float *col = cur + 8 * (q + u) + g;
            const bool in = u == 0 || two;
            split_tf32(in && s0 < S0 ? col[s0 * kCS] : 0.f, bh[u][0], bl[u][0]);
            split_tf32(in && s1 < S0 ? col[s1 * kCS] : 0.f, bh[u][1], bl[u][1]);
          }
          three_parts([&](auto P) {
#pragma unroll
            for (int m = 0; m < NM; ++m)
#pragma unroll
              for (int u = 0; u < 2; ++u)
                mma_3xtf32_part<decltype(P)::value>(d[u][m], mh[m][kk], ml[m][kk], bh[u][0], bh[u][1], bl[u][0],
                                                    bl[u][1]);
          });
        }
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (u == 1 && !two) break;
          const int c = 8 * (q + u) + 2 * t;
#pragma unroll
          for (int j = 0; j < NR; ++j) {
            const float2 y = *reinterpret_cast<const float2 *>(cur + (S0 + j) * kCS + c);
#pragma unroll
            for (int m = 0; m < NM; ++m)
#pragma unroll
              for (int e2 = 0; e2 < 2; ++e2) {
                d[u][m][2 * e2] = fmaf(mr[m][e2][j], y.x, d[u][m][2 * e2]);
                d[u][m][2 * e2 + 1] = fmaf(mr[m][e2][j], y.y, d[u][m][2 * e2 + 1]);
              }
          }
        }
        __syncwarp();  // every lane has read these columns
#pragma unroll
        for (int u = 0; u < 2; ++u) {
          if (u == 1 && !two) break;
          const int c = 8 * (q + u) + 2 * t;
#pragma unroll
          for (int m = 0; m < NM; ++m)
#pragma unroll
            for (int e2 = 0; e2 < 2; ++e2) {
              const int r = 16 * m + g + 8 * e2;
              if (r < n) *reinterpret_cast<float2 *>(cur + r * kCS + c) = make_float2(d[u][m][2 * e2], d[u][m][2 * e2 + 1]);
            }
        }
      }
      __syncwarp();  // Y_l of this chunk complete in the buffer
#pragma unroll
      for (int u = 0; u < NE; ++u) {
        const int e = lane + 32 * u, r = e >> 3, j = e & 7;
        if (r < n && j < w4) {
          const int c = c0 + 4 * j;
          const float4 y = lds4(cur + r * kCS + 4 * j);
          __stcs(reinterpret_cast<float4 *>(Yl + (size_t)r * RW + c0) + j, y);
          const bool hz = c >= N3p;
          atomicAdd(reinterpret_cast<float4 *>((hz ? a.Zh : a.Zv) + (size_t)off[r] * N3p + (hz ? c - N3p : c)), y);
        }
      }
      __syncwarp();  // every lane has read this buffer before it is refilled
    }
  }
}

template <int K>
__global__ void __launch_bounds__(kSW * 32, 4) block_dual_stream_kernel(BlockDualArgs a) {
  extern __shared__ __align__(16) float smem[];
  if (a.sc->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float *bufs = smem + warp * StreamLayout<K>::per_warp;
  const unsigned long long pol_keep = l2_evict_last(), pol_done = l2_evict_first();
  unsigned long long sweeps = 0, fo_count = 0;
  const long long step = (long long)gridDim.x * kSW;
  for (long long l = (long long)blockIdx.x * kSW + warp; l < a.dm.P; l += step)
    stream_block<K>(a, l, bufs, pol_keep, pol_done, sweeps, fo_count);
  if (lane == 0) {
    if (sweeps) atomicAdd(&a.sc->jacobi_sweeps, sweeps);
    if (fo_count) atomicAdd(&a.sc->fo_blocks, fo_count);
  }
}

// The batched solve's block duals: one work list over the blocks of every
// problem with block side K (problem i owns entries [items[i].first,
// items[i + 1].first)), taken by the warps of one persistent grid; each
// problem keeps its own sizes, step size, stop flag and statistics.
template <int K>
__global__ void __launch_bounds__(kSW * 32, 4) block_dual_stream_batch_kernel(const BatchDual *items, int n,
                                                                              long long total) {
  extern __shared__ __align__(16) float smem[];
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  float *bufs = smem + warp * StreamLayout<K>::per_warp;
  const unsigned long long pol_keep = l2_evict_last(), pol_done = l2_evict_first();
  unsigned long long sweeps = 0, fo_count = 0;
  int c = 0;
  auto flush = [&]() {
    if (lane == 0) {
      if (sweeps) atomicAdd(&items[c].a.sc->jacobi_sweeps, sweeps);
      if (fo_count) atomicAdd(&items[c].a.sc->fo_blocks, fo_count);
    }
    sweeps = fo_count = 0;
  };
  const long long step = (long long)gridDim.x * kSW;
  for (long long e = (long long)blockIdx.x * kSW + warp; e < total; e += step) {
    if (c + 1 < n && items[c + 1].first <= e) {  // a warp's entries only grow: move forward
      flush();
      while (c + 1 < n && items[c + 1].first <= e) ++c;
    }
    const BlockDualArgs &a = items[c].a;
    if (a.sc->done) continue;
    stream_block<K>(a, e - items[c].first, bufs, pol_keep, pol_done, sweeps, fo_count);
  }
  flush();
}

using BatchFn = void (*)(const BatchDual *, int, long long);
BatchFn batch_kernel(int k) {
  switch (k) {
    case 1: return block_dual_stream_batch_kernel<1>;
    case 2: return block_dual_stream_batch_kernel<2>;
    case 3: return block_dual_stream_batch_kernel<3>;
    case 4: return block_dual_stream_batch_kernel<4>;
    case 5: return block_dual_stream_batch_kernel<5>;
    default: return nullptr;
  }
}
size_t batch_smem(int k) {
  switch (k) {
    case 1: return sizeof(float) * kSW * StreamLayout<1>::per_warp;
    case 2: return sizeof(float) * kSW * StreamLayout<2>::per_warp;
    case 3: return sizeof(float) * kSW * StreamLayout<3>::per_warp;
    case 4: return sizeof(float) * kSW * StreamLayout<4>::per_warp;
    case 5: return sizeof(float) * kSW * StreamLayout<5>::per_warp;
    default: return 0;
  }
}

using KernelFn = void (*)(BlockDualArgs);

// Variants compiled (null for the others): the CUDA-core form (tc 0) for 5
// and 4 CTAs per SM; the tensor-core group form (tc 1) for 4 only (its five-
// and six-CTA variants fit in shared memory, but at 96 and 80 registers they
// spill and ran slower); the tensor-core streaming form (tc 2) for 4.
template <int K>
KernelFn kernel_k(int minb, int tc) {
  if (tc == 2) return minb == 4 ? block_dual_stream_kernel<K> : nullptr;
  if (tc) return minb == 4 ? block_dual_kernel<K, 4, true> : nullptr;
  if (minb != 5 && minb != 4) return nullptr;
  return minb == 5 ? block_dual_kernel<K, 5, false> : block_dual_kernel<K, 4, false>;
}

KernelFn kernel_for(const BdVariant &v) {
  switch (v.k) {
    case 1: return kernel_k<1>(v.minb, v.tc);
    case 2: return kernel_k<2>(v.minb, v.tc);
    case 3: return kernel_k<3>(v.minb, v.tc);
    case 4: return kernel_k<4>(v.minb, v.tc);
    case 5: return kernel_k<5>(v.minb, v.tc);
    default: return nullptr;
  }
}

template <int K, bool TC>
size_t smem_k(int rs) {
  return sizeof(float) * (yp_floats<K, TC>(rs) + kNW * gm_floats<K, TC>() + (TC ? 0 : tiles_floats<K, TC>()));
}

template <int K>
size_t smem_kt(int tc, int rs) {
  if (tc == 2) return sizeof(float) * kSW * StreamLayout<K>::per_warp;
  return tc ? smem_k<K, true>(rs) : smem_k<K, false>(rs);
}

}  // namespace

long long block_dual_w_stride(int k) {
  if (k >= kMinLargeK) return block_dual_large_w_stride(k);
  switch (k) {
    case 1: return w_floats<1>();
    case 2: return w_floats<2>();
    case 3: return w_floats<3>();
    case 4: return w_floats<4>();
    case 5: return w_floats<5>();
    default: return 0;
  }
}

// 2 N3p plus padding to 12 mod 32 words: the Gram's reads (8 rows x 4
// consecutive columns, or 8 rows x one float4, per warp access) and the
// tensor-core apply's reads (4 rows x 8 consecutive columns) spread over the
// banks (the apply's with 2-way conflicts on 4 of them).
int block_dual_row_stride(int N3p) {
  const int base = 2 * N3p;
  const int pad = ((12 - base % 32) + 32) % 32;
  return base + pad;
}

int block_dual_threads() { return kNW * 32; }

int block_dual_group() { return kNW; }

size_t block_dual_smem_bytes(const BdVariant &v, int N3p) {
  const int rs = block_dual_row_stride(N3p);
  switch (v.k) {
    case 1: return smem_kt<1>(v.tc, rs);
    case 2: return smem_kt<2>(v.tc, rs);
    case 3: return smem_kt<3>(v.tc, rs);
    case 4: return smem_kt<4>(v.tc, rs);
    case 5: return smem_kt<5>(v.tc, rs);
    default: return 0;
  }
}

bool block_dual_has(const BdVariant &v) { return kernel_for(v) != nullptr; }

// The launch limit is a property of the kernel, shared by every context and
// problem that launches it, so it is raised to the device's opt-in maximum
// (the launch's own request decides what a CTA gets) rather than to one
// problem's size, which a later, smaller problem would lower again.
cudaError_t block_dual_prepare(const BdVariant &v, size_t smem) {
  KernelFn f = kernel_for(v);
  if (!f) return cudaErrorInvalidValue;
  int dev = 0, cap = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  cudaFuncAttributes fa;
  if (e == cudaSuccess) e = cudaFuncGetAttributes(&fa, reinterpret_cast<const void *>(f));
  if (e != cudaSuccess) return e;
  const size_t dyn = (size_t)cap > fa.sharedSizeBytes ? (size_t)cap - fa.sharedSizeBytes : 0;  // minus static
  if (dyn < smem) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(reinterpret_cast<const void *>(f), cudaFuncAttributeMaxDynamicSharedMemorySize,
                              (int)dyn);
}

cudaError_t block_dual_occupancy(const BdVariant &v, size_t smem, int *ctas) {
  KernelFn f = kernel_for(v);
  if (!f) return cudaErrorInvalidValue;
  return cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas, reinterpret_cast<const void *>(f), kNW * 32, smem);
}

cudaError_t block_dual_batch_prepare(int k, int *ctas_per_sm) {
  BatchFn f = batch_kernel(k);
  if (!f) return cudaErrorInvalidValue;
  int dev = 0, cap = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  const size_t smem = batch_smem(k);
  if (e == cudaSuccess && (size_t)cap < smem) return cudaErrorInvalidValue;
  if (e == cudaSuccess) e = cudaFuncSetAttribute(f, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e == cudaSuccess) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(ctas_per_sm, f, kSW * 32, smem);
  return e;
}

cudaError_t launch_block_dual_batch(int k, const BatchDual *items, int n, long long total, int grid, cudaStream_t st) {
  BatchFn f = batch_kernel(k);
  if (!f) return cudaErrorInvalidValue;
  f<<<grid, kSW * 32, batch_smem(k), st>>>(items, n, total);
  return cudaGetLastError();
}

cudaError_t launch_block_dual(const BlockDualArgs &a, const BdVariant &v, int grid, size_t smem, cudaStream_t st) {
  KernelFn f = kernel_for(v);
  if (!f) return cudaErrorInvalidValue;
  f<<<grid, kNW * 32, smem, st>>>(a);
  return cudaGetLastError();
}

}  // namespace s3ttv
