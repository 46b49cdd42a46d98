// Evaluation of a restored cube (Sec. IV-A) and the objective value of
// Prob. (S3TTV_denoising): the reductions behind s3ttv_quality and
// s3ttv_objective.  Cubes here are the caller's plain layout [N1][N2][N3]
// (band fastest).
// Every sum accumulates in FP64.
#include <math.h>

#include "s3ttv_internal.cuh"

namespace s3ttv {
namespace {

// Per-band sums of (u - ref)^2: thread t of a block owns bands t, t + 256, ...
// and walks the block's pixels, so a warp reads consecutive bands.
__global__ void __launch_bounds__(256) band_sqerr_kernel(const float *u, const float *ref, long long P, int N3,
                                                        long long chunk, double *out) {
  const long long p0 = blockIdx.x * chunk, p1 = p0 + chunk < P ? p0 + chunk : P;
  for (int b = threadIdx.x; b < N3; b += blockDim.x) {
    double s = 0.0;
    for (long long p = p0; p < p1; ++p) {
      const double d = (double)u[p * N3 + b] - (double)ref[p * N3 + b];
      s = fma(d, d, s);
    }
    if (p1 > p0) atomicAdd(out + b, s);
  }
}

// Spectral angle at every pixel, one warp per pixel: lanes stride over the
// bands; the angle is acos of the clipped normalized inner product (pi / 2 if
// one spectrum is zero, 0 if both are).
__global__ void __launch_bounds__(256) sam_kernel(const float *u, const float *ref, long long P, int N3,
                                                 float *map, double *sum) {
  __shared__ double red[8];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double acc = 0.0;
  for (long long p = blockIdx.x * 8LL + warp; p < P; p += gridDim.x * 8LL) {
    double dot = 0.0, nu = 0.0, nr = 0.0;
    for (int b = lane; b < N3; b += 32) {
      const double x = u[p * N3 + b], y = ref[p * N3 + b];
      dot = fma(x, y, dot);
      nu = fma(x, x, nu);
      nr = fma(y, y, nr);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      dot += __shfl_xor_sync(kFull, dot, o);
      nu += __shfl_xor_sync(kFull, nu, o);
      nr += __shfl_xor_sync(kFull, nr, o);
    }
    double ang;
    if (nu > 0.0 && nr > 0.0) {
      double c = dot / (sqrt(nu) * sqrt(nr));
      c = c > 1.0 ? 1.0 : (c < -1.0 ? -1.0 : c);
      ang = acos(c);
    } else {
      ang = (nu > 0.0 || nr > 0.0) ? 1.5707963267948966 : 0.0;
    }
    if (lane == 0) {
      if (map) map[p] = (float)ang;
      acc += ang;
    }
  }
  if (lane == 0) red[warp] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w];
    atomicAdd(sum, s);
  }
}

__constant__ double c_ssim_w[kSsimTaps * kSsimTaps];

// SSIM map of band b at every pixel whose 11 x 11 window lies inside the image,
// summed per band.  Block (32 bands) x (8 pixels); weighted moments in FP64.
__global__ void __launch_bounds__(256) ssim_kernel(const float *u, const float *ref, int N1, int N2, int N3,
                                                  int b0, int nb, double *out) {
  __shared__ double red[8][32];
  const int r = kSsimTaps / 2;
  const int tb = threadIdx.x & 31, tp = threadIdx.x >> 5;
  const int b = b0 + blockIdx.x * 32 + tb;
  const int Hv = N1 - 2 * r, Wv = N2 - 2 * r;
  const long long npix = (long long)Hv * Wv;
  double acc = 0.0;
  if (b < b0 + nb) {
    for (long long q = blockIdx.y * 8LL + tp; q < npix; q += gridDim.y * 8LL) {
      const int i = (int)(q / Wv) + r, j = (int)(q % Wv) + r;
      double mx = 0.0, my = 0.0, sxx = 0.0, syy = 0.0, sxy = 0.0;
      for (int a = 0; a < kSsimTaps; ++a) {
        const float *rowx = ref + ((long long)(i + a - r) * N2 + (j - r)) * N3 + b;
        const float *rowy = u + ((long long)(i + a - r) * N2 + (j - r)) * N3 + b;
#pragma unroll
        for (int c = 0; c < kSsimTaps; ++c) {
          const double w = c_ssim_w[a * kSsimTaps + c];
          const double x = rowx[(long long)c * N3], y = rowy[(long long)c * N3];
          mx = fma(w, x, mx);
          my = fma(w, y, my);
          sxx = fma(w * x, x, sxx);
          syy = fma(w * y, y, syy);
          sxy = fma(w * x, y, sxy);
        }
      }
      sxx -= mx * mx;
      syy -= my * my;
      sxy -= mx * my;
      const double C1 = 1e-4, C2 = 9e-4;  // (0.01 L)^2, (0.03 L)^2 with L = 1
      acc += ((2.0 * mx * my + C1) * (2.0 * sxy + C2)) / ((mx * mx + my * my + C1) * (sxx + syy + C2));
    }
  }
  red[tp][tb] = acc;
  __syncthreads();
  if (tp == 0 && b < b0 + nb) {
    double s = 0.0;
    for (int w = 0; w < 8; ++w) s += red[w][tb];
    atomicAdd(out + (b - b0), s);
  }
}

// S3TTV(u) = sum_l ||X_l||_*, X_l the k^2 x 2N3 structure tensor of block l
// (eq. SSST: row a k + c is pixel ((p+a) mod N1, (q+c) mod N2), column 2b its
// D_v D_s u and 2b+1 its D_h D_s u at band b, periodic differences).  One CTA
// per block, all in FP64: the entries of X_l from the FP32 cube, the Gram
// G = X_l X_l^T accumulated in shared memory over chunks of kObjCW columns,
// then a one-sided (Hestenes) Jacobi on the rows of G (round-robin pairs, eight
// lanes per pair) until they are orthogonal: row r becomes lambda_r u_r^T, so
// sigma_r = sqrt(|row r|).  Rows below 1e-14 ||G||_F are numerical zeros.  The sigma of every block are summed into *out.
constexpr int kObjCW = 32;

__global__ void __launch_bounds__(256) objective_kernel(const float *u, int N1, int N2, int N3, int k, int stacked,
                                                       int open_s, int first_order, int parts, double tol,
                                                       int max_sweeps, double *out, unsigned *nonconv) {
  extern __shared__ double dsm[];
  const int n = stacked ? 2 * k * k : k * k, NP = n + (n & 1), W = stacked ? N3 : parts * N3;
  double *G = dsm;                 // NP x n
  double *X = dsm + (size_t)NP * n;  // n x kObjCW
  __shared__ double nrm[kMaxLargeK * kMaxLargeK];  // >= 2 kMaxStackedK^2 rows too
  __shared__ double s_fro2;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const long long L = (long long)N1 * N2;
  double total = 0.0;
  for (long long l = blockIdx.x; l < L; l += gridDim.x) {
    const int p = (int)(l / N2), q = (int)(l - (long long)p * N2);
    for (int e = tid; e < NP * n; e += 256) G[e] = 0.0;
    for (int c0 = 0; c0 < W; c0 += kObjCW) {
      __syncthreads();
      for (int e = tid; e < n * kObjCW; e += 256) {
        const int r = e / kObjCW, cc = e - r * kObjCW, col = c0 + cc;
        double x = 0.0;
        // paper layout: row r is window pixel r, column parts * b + o; stacked:
        // row 2r + o is pixel r, column b; o = 0 vertical, 1 horizontal, 2
        // spectral (SSST)
        const int pr = stacked ? r >> 1 : r, o = stacked ? r & 1 : col % parts, b = stacked ? col : col / parts;
        if (col < W && !(open_s && b == N3 - 1)) {
          const int a = pr / k, c = pr - a * k;
          const int i = (p + a) % N1, j = (q + c) % N2;
          const int i1 = i + 1 == N1 ? 0 : i + 1, j1 = j + 1 == N2 ? 0 : j + 1, b1 = b + 1 == N3 ? 0 : b + 1;
          const size_t s00 = ((size_t)i * N2 + j) * N3;
          const size_t s10 = o ? ((size_t)i * N2 + j1) * N3 : ((size_t)i1 * N2 + j) * N3;
          if (o == 2) {  // SSST: D_s u
            x = (double)u[s00 + b1] - (double)u[s00 + b];
          } else if (first_order) {  // STV, SSST: D_v u or D_h u
            x = (double)u[s10 + b] - (double)u[s00 + b];
          } else {
            const double ds0 = (double)u[s00 + b1] - (double)u[s00 + b];
            const double ds1 = (double)u[s10 + b1] - (double)u[s10 + b];
            x = ds1 - ds0;
          }
        }
        X[r * kObjCW + cc] = x;
      }
      __syncthreads();
      for (int e = tid; e < n * n; e += 256) {
        const int i = e / n, j = e - i * n;
        if (j < i) continue;
        double s = 0.0;
        for (int c = 0; c < kObjCW; ++c) s = fma(X[i * kObjCW + c], X[j * kObjCW + c], s);
        G[i * n + j] += s;
      }
    }
    __syncthreads();
    if (tid == 0) s_fro2 = 0.0;
    __syncthreads();
    {
      double f2 = 0.0;
      for (int e = tid; e < n * n; e += 256) {
        const int i = e / n, j = e - i * n;
        if (j < i) G[i * n + j] = G[j * n + i];
        const double g = G[j <= i ? j * n + i : i * n + j];
        f2 = fma(g, g, f2);
      }
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) f2 += __shfl_xor_sync(kFull, f2, o);
      if (lane == 0) atomicAdd(&s_fro2, f2);
    }
    __syncthreads();
    // rows below 1e-14 ||G||_F are numerically zero (their sigma is below
    // 1e-7 sqrt(||G||_F)): they take part in no rotation and count as zero
    const double floor2 = 1e-28 * s_fro2;
    // one-sided Jacobi on the rows of G (row NP - 1 is zero when n is odd)
    bool converged = false;
    for (int sw = 0; sw < max_sweeps && !converged; ++sw) {
      int rotated = 0;
      for (int step = 0; step < NP - 1; ++step) {
        for (int base = 0; base < NP / 2; base += 32) {
          const int i = base + (tid >> 3), gl = tid & 7;
          const bool act = i < NP / 2;
          const int pa = act ? i : 0, pb = NP - 1 - pa;
          int xa = pa - 1 + step, xb = pb - 1 + step;
          xa -= xa >= NP - 1 ? NP - 1 : 0;
          xb -= xb >= NP - 1 ? NP - 1 : 0;
          const int ra = pa == 0 ? 0 : 1 + xa, rb = 1 + xb;
          double *A = G + (size_t)ra * n, *B = G + (size_t)rb * n;
          double d = 0.0, na = 0.0, nb = 0.0;
          if (act)
            for (int c = gl; c < n; c += 8) {
              d = fma(A[c], B[c], d);
              na = fma(A[c], A[c], na);
              nb = fma(B[c], B[c], nb);
            }
#pragma unroll
          for (int o = 4; o > 0; o >>= 1) {
            d += __shfl_xor_sync(kFull, d, o);
            na += __shfl_xor_sync(kFull, na, o);
            nb += __shfl_xor_sync(kFull, nb, o);
          }
          if (act && fmin(na, nb) > floor2 && fabs(d) > tol * sqrt(na * nb)) {
            // rotation that makes rows A and B orthogonal (Hestenes)
            const double zeta = (nb - na) / (2.0 * d);
            const double t = copysign(1.0, zeta) / (fabs(zeta) + sqrt(1.0 + zeta * zeta));
            const double cs = 1.0 / sqrt(1.0 + t * t), sn = cs * t;
            for (int c = gl; c < n; c += 8) {
              const double x = A[c], y = B[c];
              A[c] = cs * x - sn * y;
              B[c] = sn * x + cs * y;
            }
            rotated = 1;
          }
        }
        __syncthreads();
      }
      converged = !__syncthreads_or(rotated);
    }
    if (!converged && tid == 0) atomicAdd(nonconv, 1u);
    for (int r = warp; r < n; r += 8) {
      double s = 0.0;
      for (int c = lane; c < n; c += 32) s = fma(G[r * n + c], G[r * n + c], s);
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kFull, s, o);
      if (lane == 0) nrm[r] = s > floor2 ? sqrt(sqrt(s)) : 0.0;  // |row r| = lambda_r; sigma_r = sqrt(lambda_r)
    }
    __syncthreads();
    if (tid == 0)
      for (int r = 0; r < n; ++r) total += nrm[r];
    __syncthreads();
  }
  if (tid == 0) atomicAdd(out, total);
}

// SSTV's objective ||D D_s u||_1 = sum |D_v D_s u| + |D_h D_s u| (periodic), FP64
__global__ void __launch_bounds__(256) sstv_l1_kernel(const float *u, int N1, int N2, int N3, double *out) {
  __shared__ double red[8];
  const long long N = (long long)N1 * N2 * N3;
  double acc = 0.0;
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < N; e += gridDim.x * 256LL) {
    const int b = (int)(e % N3);
    const long long pix = e / N3;
    const int i = (int)(pix / N2), j = (int)(pix % N2);
    const int i1 = i + 1 == N1 ? 0 : i + 1, j1 = j + 1 == N2 ? 0 : j + 1, b1 = b + 1 == N3 ? 0 : b + 1;
    const size_t p0 = (size_t)pix * N3, pv = ((size_t)i1 * N2 + j) * N3, ph = ((size_t)i * N2 + j1) * N3;
    const double ds0 = (double)u[p0 + b1] - (double)u[p0 + b];
    acc += fabs(((double)u[pv + b1] - (double)u[pv + b]) - ds0) + fabs(((double)u[ph + b1] - (double)u[ph + b]) - ds0);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(out, t);
  }
}

// HSSTV's objective: || (D_v D_s u, D_h D_s u, omega D_v u, omega D_h u) || summed
// over voxels, l1 (l12 = 0) or the l2 norm of each voxel's four entries (l12 = 1)
__global__ void __launch_bounds__(256) hsstv_norm_kernel(const float *u, int N1, int N2, int N3, double omega, int l12,
                                                        double *out) {
  __shared__ double red[8];
  const long long N = (long long)N1 * N2 * N3;
  double acc = 0.0;
  for (long long e = blockIdx.x * 256LL + threadIdx.x; e < N; e += gridDim.x * 256LL) {
    const int b = (int)(e % N3);
    const long long pix = e / N3;
    const int i = (int)(pix / N2), j = (int)(pix % N2);
    const int i1 = i + 1 == N1 ? 0 : i + 1, j1 = j + 1 == N2 ? 0 : j + 1, b1 = b + 1 == N3 ? 0 : b + 1;
    const size_t p0 = (size_t)pix * N3, pv = ((size_t)i1 * N2 + j) * N3, ph = ((size_t)i * N2 + j1) * N3;
    const double ds0 = (double)u[p0 + b1] - (double)u[p0 + b];
    const double a0 = ((double)u[pv + b1] - (double)u[pv + b]) - ds0;
    const double a1 = ((double)u[ph + b1] - (double)u[ph + b]) - ds0;
    const double a2 = omega * ((double)u[pv + b] - (double)u[p0 + b]);
    const double a3 = omega * ((double)u[ph + b] - (double)u[p0 + b]);
    acc += l12 ? sqrt(a0 * a0 + a1 * a1 + a2 * a2 + a3 * a3) : fabs(a0) + fabs(a1) + fabs(a2) + fabs(a3);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_xor_sync(kFull, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int w = 0; w < 8; ++w) t += red[w];
    atomicAdd(out, t);
  }
}

}  // namespace

cudaError_t launch_hsstv_norm(const float *u, int N1, int N2, int N3, double omega, int l12, double *out, int grid,
                              cudaStream_t st) {
  hsstv_norm_kernel<<<grid, 256, 0, st>>>(u, N1, N2, N3, omega, l12, out);
  return cudaGetLastError();
}

cudaError_t launch_sstv_l1(const float *u, int N1, int N2, int N3, double *out, int grid, cudaStream_t st) {
  sstv_l1_kernel<<<grid, 256, 0, st>>>(u, N1, N2, N3, out);
  return cudaGetLastError();
}

cudaError_t launch_band_sqerr(const float *u, const float *ref, long long P, int N3, double *out, int grid,
                              cudaStream_t st) {
  const long long chunk = (P + grid - 1) / grid;
  band_sqerr_kernel<<<(unsigned)((P + chunk - 1) / chunk), 256, 0, st>>>(u, ref, P, N3, chunk, out);
  return cudaGetLastError();
}

cudaError_t launch_sam(const float *u, const float *ref, long long P, int N3, float *map, double *sum, int grid,
                       cudaStream_t st) {
  long long g = (P + 7) / 8;
  if (g > grid) g = grid;
  sam_kernel<<<(unsigned)g, 256, 0, st>>>(u, ref, P, N3, map, sum);
  return cudaGetLastError();
}

cudaError_t launch_ssim(const float *u, const float *ref, int N1, int N2, int N3, int b0, int nb, double *out,
                        int grid, cudaStream_t st) {
  // the Gaussian window of [Wang et al. 2004]: standard deviation 1.5, 11 x 11, sum 1
  double w[kSsimTaps * kSsimTaps], tot = 0.0;
  const int r = kSsimTaps / 2;
  for (int a = 0; a < kSsimTaps; ++a)
    for (int c = 0; c < kSsimTaps; ++c) {
      const double x = a - r, y = c - r;
      w[a * kSsimTaps + c] = exp(-(x * x + y * y) / (2.0 * 1.5 * 1.5));
      tot += w[a * kSsimTaps + c];
    }
  for (double &x : w) x /= tot;
  cudaError_t e = cudaMemcpyToSymbolAsync(c_ssim_w, w, sizeof(w), 0, cudaMemcpyHostToDevice, st);
  if (e != cudaSuccess) return e;
  const long long npix = (long long)(N1 - 2 * (kSsimTaps / 2)) * (N2 - 2 * (kSsimTaps / 2));
  const int gx = (nb + 31) / 32;
  long long gy = (npix + 7) / 8;
  const long long cap = (grid + gx - 1) / gx;
  if (gy > cap) gy = cap;
  if (gy < 1) gy = 1;
  ssim_kernel<<<dim3(gx, (unsigned)gy), 256, 0, st>>>(u, ref, N1, N2, N3, b0, nb, out);
  return cudaGetLastError();
}

size_t objective_smem_bytes(int k, int stacked) {
  const int n = stacked ? 2 * k * k : k * k, NP = n + (n & 1);
  return sizeof(double) * ((size_t)NP * n + (size_t)n * kObjCW);
}

cudaError_t launch_objective(const float *u, int N1, int N2, int N3, int k, int stacked, int open_s,
                             int first_order, double *out, unsigned *nonconv, int grid, cudaStream_t st,
                             int parts) {
  const size_t smem = objective_smem_bytes(k, stacked);
  cudaError_t e = cudaFuncSetAttribute(objective_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
  if (e != cudaSuccess) return e;
  const long long L = (long long)N1 * N2;
  objective_kernel<<<(unsigned)(L < grid ? L : grid), 256, smem, st>>>(u, N1, N2, N3, k, stacked, open_s, first_order,
                                                                       parts, 1e-13, 60, out, nonconv);
  return cudaGetLastError();
}

}  // namespace s3ttv
