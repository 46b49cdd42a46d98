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
// Work decomposition: one warp owns one block at a time.  Its Y' lives in shared
// memory (rows of 2*N3p floats, padded so the row stride is 4 mod 32 words and
// the float4 reads of the Gram tiles do not conflict).  The Gram is computed in
// k x k register tiles (lane (R, S) owns G[Rk.., Sk..]).  The eigenproblem is
// solved by one-sided (Hestenes) Jacobi on the rows of G: rotating pairs of rows
// until all rows are mutually orthogonal leaves row x = lam_x u_x^T, so the
// eigenvalue is the row norm and the eigenvector its direction; no rotation
// matrix is accumulated.  Row pairs sit in lane pairs (each lane holds half of
// both rows) and move between lanes in the round-robin order, so every pair of
// rows meets once per sweep.
//
// Warm start: the rows of a block's eigenbasis change little from one pass of
// Alg. 1 to the next, so each block keeps its normalized converged rows W (one
// row per round-robin position) and the next pass starts the one-sided Jacobi
// from C0 = W G instead of G.  With W orthogonal, rows of J^T C0 that are
// mutually orthogonal are again lam_x u_x^T, so the result is the same
// decomposition; it only needs fewer sweeps.  A block whose rows did not all
// come out as nonzero directions stores a NaN marker and starts cold next time.
#include <math.h>
#include "s3ttv_internal.cuh"

namespace s3ttv {
namespace {

template <int K>
struct Shape {
  static constexpr int n = K * K;        // rows of a block (and of G)
  static constexpr int NP = (n + 1) / 2; // row pairs (a zero row when n is odd)
  static constexpr int NPOS = 2 * NP;    // round-robin positions
  static constexpr int H = (n + 1) / 2;  // half-row length held by one lane
  static constexpr int GS = n + 1;       // stride of G, M and the eigen-rows
};

__device__ __forceinline__ float4 lds4(const float *p) { return *reinterpret_cast<const float4 *>(p); }
__device__ __forceinline__ void sts4(float *p, float4 v) { *reinterpret_cast<float4 *>(p) = v; }

// 16-byte global -> shared copy that bypasses L1 (cp.async, completes at wait_all)
__device__ __forceinline__ void cp_async16(float *sdst, const float *gsrc) {
  const unsigned sa = (unsigned)__cvta_generic_to_shared(sdst);
  asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gsrc) : "memory");
}
__device__ __forceinline__ void cp_async_wait_all() {
  asm volatile("cp.async.commit_group;\n" ::: "memory");
  asm volatile("cp.async.wait_group 0;\n" ::: "memory");
}

template <int K>
__global__ void __launch_bounds__(256) block_dual_kernel(BlockDualArgs a) {
  using S = Shape<K>;
  constexpr int n = S::n, NP = S::NP, NPOS = S::NPOS, H = S::H, GS = S::GS;
  extern __shared__ __align__(16) float smem[];
  __shared__ unsigned s_sweeps;
  if (a.sc->done) return;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  if (threadIdx.x == 0) s_sweeps = 0u;
  __syncthreads();
  const int RS = a.rs;
  // per-warp slice rounded to 32 floats so every warp's Y' rows stay 16-byte aligned
  const size_t per_warp = ((size_t)n * RS + (size_t)n * GS + (size_t)NPOS * GS + 31) & ~(size_t)31;
  float *Yp = smem + warp * per_warp;
  float *Gm = Yp + (size_t)n * RS;  // G, then M
  float *Ut = Gm + n * GS;          // rows sqrt(1 - lam^-1/2) u_x^T
  const Dims dm = a.dm;
  const int N3p = dm.N3p, C4 = N3p >> 2, W4 = 2 * C4;
  const long long L = dm.P;
  const float gY = a.gY;

  for (long long l = (long long)blockIdx.x * a.warps + warp; l < L; l += (long long)gridDim.x * a.warps) {
    const int p = (int)(l / dm.N2), q = (int)(l - (long long)p * dm.N2);
    float *Yl = a.Y + (size_t)l * n * 2 * N3p;

    // ---- 1. Y' = Y + gamma_Y X,  X = P_l D D_s ubar (eq. rewrite_Lu) ----
    for (int idx = lane; idx < n * W4; idx += 32) {
      const int r = idx / W4, c4 = idx - r * W4;
      cp_async16(Yp + (size_t)r * RS + (c4 << 2), Yl + (size_t)r * 2 * N3p + (c4 << 2));
    }
    cp_async_wait_all();
    __syncwarp();
#pragma unroll 1
    for (int r = 0; r < n; ++r) {
      const int ra = r / K, rc = r - ra * K;
      int i = p + ra;
      if (i >= dm.N1) i -= dm.N1;
      int j = q + rc;
      if (j >= dm.N2) j -= dm.N2;
      const int i1 = (i + 1 == dm.N1) ? 0 : i + 1, j1 = (j + 1 == dm.N2) ? 0 : j + 1;
      const float *u00 = a.ubar + ((size_t)i * dm.N2 + j) * N3p;
      const float *uv = a.ubar + ((size_t)i1 * dm.N2 + j) * N3p;
      const float *uh = a.ubar + ((size_t)i * dm.N2 + j1) * N3p;
      for (int c4 = lane; c4 < W4; c4 += 32) {
        const bool hz = c4 >= C4;
        const int b0 = (hz ? c4 - C4 : c4) << 2;
        const float *un = hz ? uh : uv;
        const float4 q0 = __ldg(reinterpret_cast<const float4 *>(u00 + b0));
        const float4 q1 = __ldg(reinterpret_cast<const float4 *>(un + b0));
        const int bw = (b0 + 4 < dm.N3) ? b0 + 4 : 0;
        const float e0[5] = {q0.x, q0.y, q0.z, q0.w, __ldg(u00 + bw)};
        const float e1[5] = {q1.x, q1.y, q1.z, q1.w, __ldg(un + bw)};
        const float w0 = __ldg(u00), w1 = __ldg(un);  // band 0, the periodic successor of N3-1
        float xs[4];
#pragma unroll
        for (int e = 0; e < 4; ++e) {
          const int b = b0 + e;
          const float n0 = (b + 1 == dm.N3) ? w0 : e0[e + 1];
          const float n1 = (b + 1 == dm.N3) ? w1 : e1[e + 1];
          // (D_v D_s ubar) = D_s ubar at the next pixel minus D_s ubar here
          xs[e] = (b < dm.N3) ? ((n1 - e1[e]) - (n0 - e0[e])) : 0.f;
        }
        float *dst = Yp + (size_t)r * RS + (c4 << 2);
        float4 y = lds4(dst);
        y.x = fmaf(gY, xs[0], y.x);
        y.y = fmaf(gY, xs[1], y.y);
        y.z = fmaf(gY, xs[2], y.z);
        y.w = fmaf(gY, xs[3], y.w);
        sts4(dst, y);
      }
    }
    __syncwarp();

    // ---- 2. G = Y' Y'^T in k x k register tiles ----
    if (lane < n) {
      const int R = lane / K, Sx = lane - R * K;
      float acc[K][K];
#pragma unroll
      for (int x = 0; x < K; ++x)
#pragma unroll
        for (int y = 0; y < K; ++y) acc[x][y] = 0.f;
      const float *pa = Yp + (size_t)(R * K) * RS;
      const float *pb = Yp + (size_t)(Sx * K) * RS;
#pragma unroll 2
      for (int c = 0; c < 2 * N3p; c += 4) {
        float4 va[K], vb[K];
#pragma unroll
        for (int x = 0; x < K; ++x) va[x] = lds4(pa + (size_t)x * RS + c);
#pragma unroll
        for (int y = 0; y < K; ++y) vb[y] = lds4(pb + (size_t)y * RS + c);
#pragma unroll
        for (int x = 0; x < K; ++x)
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
#pragma unroll
      for (int x = 0; x < K; ++x)
#pragma unroll
        for (int y = 0; y < K; ++y) Gm[(R * K + x) * GS + Sx * K + y] = acc[x][y];
    }
    __syncwarp();

    // ---- 3. one-sided Jacobi on the rows of G (or of C0 = W G) ----
    // Positions 0..NPOS-1 hold the rows; lane pair i (lanes 2i, 2i+1, one half of
    // each row) holds positions (2i, 2i+1) on even steps and (2i+1, 2i+2) on odd
    // steps (the odd-even ordering: neighbours rotate, then trade places, so every
    // pair of rows meets once in NPOS steps).  Between steps one row per lane
    // moves one lane pair along a ring; on odd steps the last lane pair holds
    // (NPOS-1, 0), which do not meet there.
    const int pi = lane >> 1, hf = lane & 1;
    const bool act = pi < NP;
    const int src_r = act ? (pi + 1 == NP ? hf : lane + 2) : lane;            // right neighbour (ring)
    const int src_l = act ? (pi == 0 ? 2 * (NP - 1) + hf : lane - 2) : lane;  // left neighbour (ring)
    float A[H], B[H];
    const float *Wl = a.W ? a.W + (size_t)l * a.w_stride : nullptr;
    const bool warm = a.warm && Wl && !(Wl[0] != Wl[0]);  // NaN marks "start cold"
    if (warm) {
      // C0 = W G: rows 2i, 2i+1 of W times G, this lane's half of the columns
      float wa[n], wb[n];
#pragma unroll
      for (int kk = 0; kk < n; ++kk) {
        wa[kk] = act ? Wl[(2 * pi) * n + kk] : 0.f;
        wb[kk] = act ? Wl[(2 * pi + 1) * n + kk] : 0.f;
      }
#pragma unroll
      for (int e = 0; e < H; ++e) {
        const int col = hf * H + e;
        float sa = 0.f, sb = 0.f;
        if (col < n) {
#pragma unroll
          for (int kk = 0; kk < n; ++kk) {
            const float g = Gm[kk * GS + col];
            sa = fmaf(wa[kk], g, sa);
            sb = fmaf(wb[kk], g, sb);
          }
        }
        A[e] = sa;
        B[e] = sb;
      }
    } else {
      const int rA = 2 * pi, rB = 2 * pi + 1;
#pragma unroll
      for (int e = 0; e < H; ++e) {
        const int col = hf * H + e;
        A[e] = (act && rA < n && col < n) ? Gm[rA * GS + col] : 0.f;
        B[e] = (act && rB < n && col < n) ? Gm[rB * GS + col] : 0.f;
      }
    }
    // squared row norms, tracked through the rotations and refreshed every sweep
    float nA, nB;
    auto refresh = [&]() {
      float x = 0.f, y = 0.f;
#pragma unroll
      for (int e = 0; e < H; ++e) {
        x = fmaf(A[e], A[e], x);
        y = fmaf(B[e], B[e], y);
      }
      nA = x + __shfl_xor_sync(kFull, x, 1);
      nB = y + __shfl_xor_sync(kFull, y, 1);
    };
    refresh();
    float fro = hf == 0 ? nA + nB : 0.f;
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) fro += __shfl_xor_sync(kFull, fro, o);
    // rows below 1e-6 ||G||_F are numerical zeros: rotating them changes any
    // other row's direction by less than 1e-6
    const float floor2 = 1e-12f * fro;
    const float tol2 = a.tol * a.tol;
    bool rotated = false;
    // One step: the pair (A, B) meets if `meets`; it is rotated to orthogonality
    // when needed, then the rows trade places.  A pair that does not meet keeps
    // its places (B's sign flips, which changes nothing the solver uses).
    auto step = [&](bool meets) {
      float apq = 0.f;
#pragma unroll
      for (int e = 0; e < H; ++e) apq = fmaf(A[e], B[e], apq);
      apq += __shfl_xor_sync(kFull, apq, 1);
      float c = 0.f, sn = 1.f, dn = 0.f;
      if (meets) {
        c = 1.f;
        sn = 0.f;
        if (fminf(nA, nB) > floor2 && apq * apq > tol2 * nA * nB) {
          const float zeta = __fdividef(nB - nA, 2.f * apq);
          const float tt = copysignf(__fdividef(1.f, fabsf(zeta) + sqrtf(fmaf(zeta, zeta, 1.f))), zeta);
          c = rsqrtf(fmaf(tt, tt, 1.f));
          sn = c * tt;
          dn = tt * apq;
          rotated = true;
        }
      }
#pragma unroll
      for (int e = 0; e < H; ++e) {
        const float x = A[e], y = B[e];
        A[e] = fmaf(sn, x, c * y);   // rotated B row, now at A's position
        B[e] = fmaf(c, x, -sn * y);  // rotated A row, now at B's position
      }
      const float oA = nA;
      nA = meets ? nB + dn : nA;
      nB = meets ? oA - dn : nB;
    };
    bool converged = false;
    int sweeps = 0;
    for (int sw = 0; sw < a.max_sweeps; ++sw) {
      rotated = false;
      if (sw) refresh();
#pragma unroll 1
      for (int sp = 0; sp < NPOS / 2; ++sp) {
        step(act);
        if constexpr (NP > 1) {  // even -> odd: keep position 2i+1, take 2i+2 from the right
#pragma unroll
          for (int e = 0; e < H; ++e) {
            const float recv = __shfl_sync(kFull, A[e], src_r);
            A[e] = B[e];
            B[e] = recv;
          }
          const float rn = __shfl_sync(kFull, nA, src_r);
          nA = nB;
          nB = rn;
        }
        step(act && pi != NP - 1);
        if constexpr (NP > 1) {  // odd -> even: keep position 2i+1, take 2i from the left
#pragma unroll
          for (int e = 0; e < H; ++e) {
            const float recv = __shfl_sync(kFull, B[e], src_l);
            B[e] = A[e];
            A[e] = recv;
          }
          const float ln = __shfl_sync(kFull, nB, src_l);
          nB = nA;
          nA = ln;
        }
      }
      ++sweeps;
      if (!__any_sync(kFull, rotated)) {
        converged = true;
        break;
      }
    }
    if (lane == 0) {
      if (!converged) atomicAdd(&a.sc->jacobi_fail, 1u);
      atomicAdd(&s_sweeps, (unsigned)sweeps);
    }

    // ---- 4. eigen-rows: lam = ||row||, keep sqrt(1 - lam^-1/2) row / lam ----
    {
      refresh();
      const float lA = sqrtf(nA), lB = sqrtf(nB);
      const float sA = lA > 1.f ? sqrtf(1.f - rsqrtf(lA)) / lA : 0.f;
      const float sB = lB > 1.f ? sqrtf(1.f - rsqrtf(lB)) / lB : 0.f;
      if (act) {
#pragma unroll
        for (int e = 0; e < H; ++e) {
          const int col = hf * H + e;
          if (col < n) {
            Ut[(2 * pi) * GS + col] = A[e] * sA;
            Ut[(2 * pi + 1) * GS + col] = B[e] * sB;
          }
        }
      }
      if (a.W) {
        // warm state for the next pass: the rows, normalized; all but the
        // NPOS - n zero rows must be nonzero directions, else mark the block cold
        const unsigned zero_rows = __popc(__ballot_sync(kFull, act && hf == 0 && nA <= floor2)) +
                                   __popc(__ballot_sync(kFull, act && hf == 0 && nB <= floor2));
        float *Ww = a.W + (size_t)l * a.w_stride;
        __syncwarp();  // every lane has read Wl[0] above
        if (zero_rows > (unsigned)(NPOS - n)) {
          if (lane == 0) Ww[0] = __int_as_float(0x7fc00000);
        } else if (act) {
          const float iA = nA > floor2 ? rsqrtf(nA) : 0.f, iB = nB > floor2 ? rsqrtf(nB) : 0.f;
#pragma unroll
          for (int e = 0; e < H; ++e) {
            const int col = hf * H + e;
            if (col < n) {
              Ww[(2 * pi) * n + col] = A[e] * iA;
              Ww[(2 * pi + 1) * n + col] = B[e] * iB;
            }
          }
        }
      }
    }
    __syncwarp();

    // ---- 5. M = I - Ut^T Ut (symmetric, written into G's space) ----
    if (lane < n) {
      const int R = lane / K, Sx = lane - R * K;
      float acc[K][K];
#pragma unroll
      for (int x = 0; x < K; ++x)
#pragma unroll
        for (int y = 0; y < K; ++y) acc[x][y] = 0.f;
#pragma unroll 2
      for (int xr = 0; xr < NPOS; ++xr) {
        float ua[K], ub[K];
#pragma unroll
        for (int x = 0; x < K; ++x) ua[x] = Ut[xr * GS + R * K + x];
#pragma unroll
        for (int y = 0; y < K; ++y) ub[y] = Ut[xr * GS + Sx * K + y];
#pragma unroll
        for (int x = 0; x < K; ++x)
#pragma unroll
          for (int y = 0; y < K; ++y) acc[x][y] = fmaf(ua[x], ub[y], acc[x][y]);
      }
#pragma unroll
      for (int x = 0; x < K; ++x)
#pragma unroll
        for (int y = 0; y < K; ++y) {
          const int r = R * K + x, s = Sx * K + y;
          Gm[r * GS + s] = (r == s ? 1.f : 0.f) - acc[x][y];
        }
    }
    __syncwarp();

    // ---- 6. Y = M Y', written back, and Z += P_l^T Y ----
#pragma unroll 1
    for (int c4 = lane; c4 < W4; c4 += 32) {
      const bool hz = c4 >= C4;
      const int b0 = (hz ? c4 - C4 : c4) << 2;
      float *Zo = hz ? a.Zh : a.Zv;
#pragma unroll 1
      for (int R = 0; R < K; ++R) {
        float4 acc[K];
#pragma unroll
        for (int x = 0; x < K; ++x) acc[x] = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll 5
        for (int s = 0; s < n; ++s) {
          const float4 y = lds4(Yp + (size_t)s * RS + (c4 << 2));
          const float *mrow = Gm + s * GS + R * K;  // M[s][R*K + x] = M[R*K + x][s]
#pragma unroll
          for (int x = 0; x < K; ++x) {
            const float m = mrow[x];
            acc[x].x = fmaf(m, y.x, acc[x].x);
            acc[x].y = fmaf(m, y.y, acc[x].y);
            acc[x].z = fmaf(m, y.z, acc[x].z);
            acc[x].w = fmaf(m, y.w, acc[x].w);
          }
        }
        int i = p + R;
        if (i >= dm.N1) i -= dm.N1;
#pragma unroll
        for (int x = 0; x < K; ++x) {
          const int r = R * K + x;
          __stcs(reinterpret_cast<float4 *>(Yl + (size_t)r * 2 * N3p) + c4, acc[x]);
          int j = q + x;
          if (j >= dm.N2) j -= dm.N2;
          atomicAdd(reinterpret_cast<float4 *>(Zo + ((size_t)i * dm.N2 + j) * N3p + b0), acc[x]);
        }
      }
    }
    __syncwarp();
  }
  __syncthreads();
  if (threadIdx.x == 0 && s_sweeps) atomicAdd(&a.sc->jacobi_sweeps, (unsigned long long)s_sweeps);
}

template <int K>
cudaError_t launch_k(const BlockDualArgs &a, int grid, size_t smem, cudaStream_t st) {
  block_dual_kernel<K><<<grid, a.warps * 32, smem, st>>>(a);
  return cudaGetLastError();
}

template <int K>
cudaError_t prepare_k(size_t smem) {
  return cudaFuncSetAttribute(block_dual_kernel<K>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
}

}  // namespace

long long block_dual_w_stride(int k) {
  const int n = k * k, npos = 2 * ((n + 1) / 2);
  return ((long long)npos * n + 3) & ~3ll;
}

int block_dual_row_stride(int N3p) {
  const int base = 2 * N3p;
  const int pad = ((4 - base % 32) + 32) % 32;
  return base + pad;
}

size_t block_dual_smem_per_warp(int k, int rs) {
  const int n = k * k, np = (n + 1) / 2, gs = n + 1;
  const size_t floats = ((size_t)n * rs + (size_t)n * gs + (size_t)(2 * np) * gs + 31) & ~(size_t)31;
  return sizeof(float) * floats;
}

cudaError_t block_dual_prepare(int k, size_t smem) {
  switch (k) {
    case 1: return prepare_k<1>(smem);
    case 2: return prepare_k<2>(smem);
    case 3: return prepare_k<3>(smem);
    case 4: return prepare_k<4>(smem);
    case 5: return prepare_k<5>(smem);
    default: return cudaErrorInvalidValue;
  }
}

cudaError_t launch_block_dual(const BlockDualArgs &a, int k, int grid, size_t smem, cudaStream_t st) {
  switch (k) {
    case 1: return launch_k<1>(a, grid, smem, st);
    case 2: return launch_k<2>(a, grid, smem, st);
    case 3: return launch_k<3>(a, grid, smem, st);
    case 4: return launch_k<4>(a, grid, smem, st);
    case 5: return launch_k<5>(a, grid, smem, st);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace s3ttv
