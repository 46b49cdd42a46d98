// Alg. 1 steps 8-11 once more, in FP64, for the blocks whose FP32 eigen-solve
// reached its sweep cap.  The block-dual kernels queue such a block (its index
// in BlockDualArgs::fb_list, the count in Scalars::fb_count), leave Y' in Y_l
// and add nothing to Z for it; this kernel then, per queued block:
//   G = Y' Y'^T in FP64 (Y' streamed by column chunks);
//   one-sided (Hestenes) Jacobi on the rows of G in FP64 (round-robin pairs,
//   tolerance 1e-13, numerical-zero floor 1e-14 ||G||_F, at most 80 sweeps),
//   which leaves row x = lam_x u_x^T;
//   Ut rows sqrt(1 - lam_x^-1/2) u_x for lam_x > 1 (0 otherwise), so that
//   Y_l = M Y' = Y' - Ut^T (Ut Y')   (M = I - Ut^T Ut, the singular values of
//   Y' clipped at 1, as in the FP32 kernels), formed chunk by chunk;
//   Y_l stored, Z += P_l^T Y_l, and the block's warm-start rows marked cold.
// One CTA per queued block (a grid-stride loop over the queue); when the queue
// is empty every CTA returns at once.  A block the FP64 solve does not settle
// either is counted in Scalars::jacobi_fail and applied as it stands.
#include <math.h>

#include "s3ttv_internal.cuh"

namespace s3ttv {
namespace {

constexpr int kFbThreads = 256;
constexpr int kFbWarps = kFbThreads / 32;
constexpr int kFbCW = 16;         // columns of Y' per chunk
constexpr int kFbMaxSweeps = 80;
constexpr unsigned kFull = 0xffffffffu;

struct FbLayout {
  int n, np;
  size_t c, x, t, nrm, pix, total_bytes;  // double offsets (pix: int offset after nrm)
};

__host__ __device__ inline FbLayout fb_layout(int n) {
  FbLayout L;
  L.n = n;
  L.np = n + (n & 1);
  L.c = 0;                                  // rows of C (np x n): G, then Ut
  L.x = L.c + (size_t)L.np * n;             // a chunk of Y' (np x kFbCW)
  L.t = L.x + (size_t)L.np * kFbCW;         // Ut times the chunk (np x kFbCW)
  L.nrm = L.t + (size_t)L.np * kFbCW;       // squared row norms (np)
  L.pix = L.nrm + L.np;                     // pixel of each row (np ints)
  L.total_bytes = sizeof(double) * L.pix + sizeof(int) * L.np;
  return L;
}

__device__ __forceinline__ double warp_sum(double v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(kFull, v, o);
  return v;
}

// k, stacked (rows 2r, 2r + 1: D_v, D_h parts of window pixel r) and parts
// (paper layout: 2, or SSST's 3 parts of N3p bands per row) as in the FP32 kernels
__global__ void __launch_bounds__(kFbThreads) fallback_kernel(BlockDualArgs a, int k, int stacked, int parts) {
  extern __shared__ __align__(16) double fsm[];
  if (a.sc->done) return;
  const unsigned queued = a.sc->fb_count;
  const unsigned cnt = queued < (unsigned)a.fb_cap ? queued : (unsigned)a.fb_cap;
  if (blockIdx.x == 0 && threadIdx.x == 0 && cnt) atomicAdd(&a.sc->fb_total, cnt);
  if (blockIdx.x >= cnt) return;
  const int n = stacked ? 2 * k * k : k * k;
  const FbLayout L = fb_layout(n);
  const int NP = L.np;
  double *C = fsm + L.c, *X = fsm + L.x, *T = fsm + L.t, *nrm = fsm + L.nrm;
  int *pix = reinterpret_cast<int *>(fsm + L.pix);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const Dims dm = a.dm;
  const int N3p = dm.N3p, W = stacked ? N3p : parts * N3p;

  for (unsigned qi = blockIdx.x; qi < cnt; qi += gridDim.x) {
    const long long l = a.fb_list[qi];
    float *Yl = a.Y + (size_t)l * n * W;
    if (tid < n) {
      const int p = (int)(l / dm.N2), q = (int)(l - (long long)p * dm.N2);
      const int pr = stacked ? tid >> 1 : tid;
      const int ra = pr / k, rc = pr - ra * k;
      int i = p + ra;
      if (i >= dm.N1) i -= dm.N1;
      int j = q + rc;
      if (j >= dm.N2) j -= dm.N2;
      pix[tid] = i * dm.N2 + j;
    }
    for (int e = tid; e < NP * n; e += kFbThreads) C[e] = 0.0;
    __syncthreads();

    // ---- G = Y' Y'^T (upper triangle, then mirrored) ----
    for (int c0 = 0; c0 < W; c0 += kFbCW) {
      for (int e = tid; e < n * kFbCW; e += kFbThreads) {
        const int r = e / kFbCW, cc = e - r * kFbCW, col = c0 + cc;
        X[e] = col < W ? (double)Yl[(size_t)r * W + col] : 0.0;
      }
      __syncthreads();
      for (int e = tid; e < n * n; e += kFbThreads) {
        const int i = e / n, j = e - i * n;
        if (j < i) continue;
        double s = 0.0;
#pragma unroll
        for (int c = 0; c < kFbCW; ++c) s = fma(X[i * kFbCW + c], X[j * kFbCW + c], s);
        C[i * n + j] += s;
      }
      __syncthreads();
    }
    for (int e = tid; e < n * n; e += kFbThreads) {
      const int i = e / n, j = e - i * n;
      if (j < i) C[i * n + j] = C[j * n + i];
    }
    __syncthreads();

    // ---- one-sided Jacobi on the rows of C = G ----
    auto norms = [&]() {
      for (int r = warp; r < NP; r += kFbWarps) {
        double s = 0.0;
        for (int c = lane; c < n; c += 32) s = fma(C[r * n + c], C[r * n + c], s);
        s = warp_sum(s);
        if (lane == 0) nrm[r] = s;
      }
      __syncthreads();
    };
    norms();
    double fro = 0.0;  // ||G||_F^2, the same sum in every thread
    for (int r = 0; r < NP; ++r) fro += nrm[r];
    const double floor2 = 1e-28 * fro, tol2 = 1e-26;
    __syncthreads();  // every thread has read nrm before the first rotation updates it
    bool converged = false;
    for (int sw = 0; sw < kFbMaxSweeps; ++sw) {
      if (sw) norms();
      int rotated = 0;
      for (int step = 0; step < NP - 1; ++step) {
        for (int pi = warp; pi < NP / 2; pi += kFbWarps) {  // warp-uniform
          // round robin: position 0 fixed, positions 1..NP-1 turn by one each step
          const int pa = pi, pb = NP - 1 - pi;
          int xa = pa - 1 + step, xb = pb - 1 + step;
          xa -= xa >= NP - 1 ? NP - 1 : 0;
          xb -= xb >= NP - 1 ? NP - 1 : 0;
          const int ra = pa == 0 ? 0 : 1 + xa, rb = 1 + xb;
          double d = 0.0;
          for (int c = lane; c < n; c += 32) d = fma(C[ra * n + c], C[rb * n + c], d);
          d = warp_sum(d);
          const double nA = nrm[ra], nB = nrm[rb];
          if (fmin(nA, nB) > floor2 && d * d > tol2 * nA * nB) {
            // tan 2 theta = 2 d / (nB - nA), |theta| <= pi / 4
            const double x = nB - nA, y = 2.0 * d;
            const double r = sqrt(fma(x, x, y * y));
            const double cs = sqrt(0.5 * (1.0 + fabs(x) / r));
            const double sn = copysign(1.0, x) * y / (2.0 * r * cs);
            for (int c = lane; c < n; c += 32) {
              const double u = C[ra * n + c], v = C[rb * n + c];
              C[ra * n + c] = cs * u - sn * v;
              C[rb * n + c] = sn * u + cs * v;
            }
            __syncwarp();  // every lane has read nrm[ra], nrm[rb]
            if (lane == 0) {
              const double t = sn / cs;
              nrm[ra] = nA - t * d;
              nrm[rb] = nB + t * d;
            }
            rotated = 1;
          }
        }
        __syncthreads();
      }
      if (!__syncthreads_or(rotated)) {
        converged = true;
        break;
      }
    }
    norms();
    if (!converged && tid == 0) atomicAdd(&a.sc->jacobi_fail, 1u);

    // ---- Ut rows in place: sqrt(1 - lam^-1/2) u for lam = ||row|| > 1 ----
    for (int r = warp; r < NP; r += kFbWarps) {
      const double nr = nrm[r], lam = sqrt(nr);
      const double w = lam > 1.0 ? sqrt(1.0 - 1.0 / sqrt(lam)) / lam : 0.0;  // / ||row|| = / lam
      for (int c = lane; c < n; c += 32) C[r * n + c] *= w;
    }
    __syncthreads();

    // ---- Y_l = Y' - Ut^T (Ut Y') by chunks; Z += P_l^T Y_l ----
    for (int c0 = 0; c0 < W; c0 += kFbCW) {
      for (int e = tid; e < n * kFbCW; e += kFbThreads) {
        const int r = e / kFbCW, cc = e - r * kFbCW, col = c0 + cc;
        X[e] = col < W ? (double)Yl[(size_t)r * W + col] : 0.0;
      }
      __syncthreads();
      for (int e = tid; e < NP * kFbCW; e += kFbThreads) {
        const int x = e / kFbCW, cc = e - x * kFbCW;
        double s = 0.0;
        for (int r = 0; r < n; ++r) s = fma(C[x * n + r], X[r * kFbCW + cc], s);
        T[e] = s;
      }
      __syncthreads();
      for (int e = tid; e < n * kFbCW; e += kFbThreads) {
        const int r = e / kFbCW, cc = e - r * kFbCW, col = c0 + cc;
        if (col >= W) continue;
        double s = X[e];
        for (int x = 0; x < NP; ++x) s = fma(-C[x * n + r], T[x * kFbCW + cc], s);
        const float y = (float)s;
        Yl[(size_t)r * W + col] = y;
        const int part = stacked ? (r & 1) : col / N3p;
        const int band = stacked ? col : col - part * N3p;
        if (band < dm.N3) {
          float *Z = part == 0 ? a.Zv : (part == 1 ? a.Zh : a.Zs);
          atomicAdd(Z + (size_t)pix[r] * N3p + band, y);
        }
      }
      __syncthreads();
    }
    if (a.W && tid == 0) a.W[(size_t)l * a.w_stride] = __int_as_float(0x7fc00000);  // start cold next pass
  }
}

}  // namespace

size_t fallback_smem_bytes(int n) { return fb_layout(n).total_bytes; }

// The attribute is set to the device's whole opt-in shared memory, not to smem:
// contexts with different block sizes share the kernel (the batched form), and
// a smaller setting made for one would make the launches of another fail.
cudaError_t fallback_prepare(size_t smem) {
  int dev = 0, cap = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e == cudaSuccess) e = cudaDeviceGetAttribute(&cap, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
  if (e != cudaSuccess) return e;
  if (smem > (size_t)cap) return cudaErrorInvalidValue;
  return cudaFuncSetAttribute(fallback_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, cap);
}

cudaError_t launch_fallback(const BlockDualArgs &a, int k, int stacked, int parts, int grid, size_t smem,
                            cudaStream_t st) {
  fallback_kernel<<<grid, kFbThreads, smem, st>>>(a, k, stacked, parts);
  return cudaGetLastError();
}

}  // namespace s3ttv
